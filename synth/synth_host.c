/*
 * synth_host.c — host side of the seeded input generators (see synth.h).
 * Dense tensors are in dimensional order: entry (i_0, ..., i_{m-1}) sits at
 * offset sum_k i_k n^k (mode 0 fastest).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include "synth.h"

/* Philox on explicit counters (used by the known-answer tests). */
void synth_philox_batch(const uint32_t* ctr, const uint32_t* key, int64_t count, uint32_t* out)
{
    for (int64_t t = 0; t < count; ++t) synth_philox4x32_10(ctr + 4 * t, key, out + 4 * t);
}

/* Dense symmetric Uniform(-1,1) tensor of order m, dimension n, FP64. */
void synth_sym_uniform_dense_f64(int m, int64_t n, uint64_t seed, double* out)
{
    int64_t total = 1;
    for (int a = 0; a < m; ++a) total *= n;
#pragma omp parallel for schedule(static)
    for (int64_t lin = 0; lin < total; ++lin) {
        int64_t idx[16];
        int64_t r = lin;
        for (int a = 0; a < m; ++a) { idx[a] = r % n; r /= n; }
        out[lin] = synth_uniform_pm1(seed, synth_sym_key(idx, m, n));
    }
}

/* Values for an explicit list of index tuples idx[count][m]. */
void synth_sym_uniform_values(int m, int64_t n, uint64_t seed, const int64_t* idx, int64_t count, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t) out[t] = synth_uniform_pm1(seed, synth_sym_key(idx + (int64_t)m * t, m, n));
}

/* Gaussian N(0, scale^2) matrix entries by Box-Muller on Philox words;
 * entry t uses counter (t, 0, 1, 0) and key (seed, 1). */
void synth_gaussian(uint64_t seed, int64_t count, double scale, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t) {
        uint32_t ctr[4] = {(uint32_t)t, (uint32_t)((uint64_t)t >> 32), 1u, 0u};
        uint32_t k[2] = {(uint32_t)seed, 1u};
        uint32_t o[4];
        synth_philox4x32_10(ctr, k, o);
        double u1 = ((double)o[0] + 0.5) * (1.0 / 4294967296.0);
        double u2 = ((double)o[1] + 0.5) * (1.0 / 4294967296.0);
        out[t] = scale * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    }
}

/* Dense rank-R symmetric tensor sum_r lambda_r a_r^{(x)m}; vecs is R x n
 * row-major (a_r = vecs[r*n : (r+1)*n]). */
void synth_rank_r_dense(int m, int64_t n, int R, const double* lambdas, const double* vecs, double* out)
{
    int64_t total = 1;
    for (int a = 0; a < m; ++a) total *= n;
#pragma omp parallel for schedule(static)
    for (int64_t lin = 0; lin < total; ++lin) {
        int64_t idx[16];
        int64_t r = lin;
        for (int a = 0; a < m; ++a) { idx[a] = r % n; r /= n; }
        double acc = 0.0;
        for (int q = 0; q < R; ++q) {
            double prod = lambdas[q];
            for (int a = 0; a < m; ++a) prod *= vecs[(int64_t)q * n + idx[a]];
            acc += prod;
        }
        out[lin] = acc;
    }
}
