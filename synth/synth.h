/*
 * synth.h — seeded synthetic inputs for sttsm tests and benchmarks.
 *
 * This module is shared by the FP64 oracle (test infrastructure) and by the
 * GPU tests/benchmark.  It holds no arithmetic of the method itself: only a
 * counter-based random generator and the map from an index tuple to a draw.
 *
 * Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), restated from its published
 * definition: two 32x32->64 multiplies per round with the constants
 * 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85,
 * ten rounds, the key bumped before every round but the first.
 *
 * Symmetric draws: the value of entry (i_0, ..., i_{m-1}) of an order-m,
 * dimension-n symmetric tensor depends only on the multiset of its indices.
 * The indices are sorted ascending (s_0 <= ... <= s_{m-1}) and keyed as the
 * mixed-radix number key = sum_k s_k n^k; the draw is word 0 of
 * Philox(counter = (key_lo, key_hi, 0, 0), key = (seed, 0)), mapped to
 * alpha = (2 * (w >> 8) + 1) / 2^24 - 1, an odd multiple of 2^-24 in (-1, 1).
 * Every such value is exact in FP32, so FP32 and FP64 inputs hold the same
 * numbers.
 */
#ifndef SYNTH_H
#define SYNTH_H

#include <stdint.h>

#if defined(__CUDACC__)
#define SYNTH_HD __host__ __device__ __forceinline__
#else
#define SYNTH_HD static inline
#endif

SYNTH_HD void synth_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform(-1,1) draw for a (pre-computed) key. Exact in FP32 and FP64. */
SYNTH_HD double synth_uniform_pm1(uint64_t seed, uint64_t key)
{
    uint32_t ctr[4] = {(uint32_t)key, (uint32_t)(key >> 32), 0u, 0u};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    synth_philox4x32_10(ctr, k, o);
    int64_t num = 2 * (int64_t)(o[0] >> 8) + 1 - ((int64_t)1 << 24);
    return (double)num * (1.0 / 16777216.0);
}

/* Key of an index tuple: sort ascending (insertion sort, m <= 16), then
 * mixed radix in base n. */
SYNTH_HD uint64_t synth_sym_key(const int64_t* idx, int m, int64_t n)
{
    int64_t s[16];
    for (int a = 0; a < m; ++a) s[a] = idx[a];
    for (int a = 1; a < m; ++a) {
        int64_t v = s[a];
        int c = a - 1;
        while (c >= 0 && s[c] > v) { s[c + 1] = s[c]; --c; }
        s[c + 1] = v;
    }
    uint64_t key = 0, w = 1;
    for (int a = 0; a < m; ++a) { key += (uint64_t)s[a] * w; w *= (uint64_t)n; }
    return key;
}

#endif
