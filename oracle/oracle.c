/*
 * oracle.c — plain, slow FP64 CPU oracle for sttsm on symmetric tensors.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load or call this code.  It shares no
 * code, header, table or helper with the GPU library, and the GPU library
 * never calls it.
 *
 * Paper: Schatz, Low, van de Geijn, Kolda, "Exploiting Symmetry in Tensors
 * for High Performance: Multiplication with Symmetric Tensors" (arXiv
 * 1301.7744).
 *
 * Conventions (Sec. 2.1, App. A):
 *   - indices are 0-based; A has order m and dimension n in every mode;
 *   - dense tensors are in "dimensional order": entry (i_0, ..., i_{m-1})
 *     is at offset sum_k i_k n^k (mode 0 fastest, the extension of
 *     column-major order named in App. A);
 *   - X is p x n with chi_{j,i} stored column-major at X[j + i*p].
 *
 * What is pinned, and by what (see tests/test_oracle_pins.py):
 *   oracle_sttsm_bruteforce  — rank-R closed form, m=2 X A X^T, identity,
 *                              diagonal and selection X, symmetry of C;
 *   oracle_ttm_chain         — equals brute force on small cases, and the
 *                              same closed forms at larger sizes;
 *   oracle_sttsm_entries     — equals the chain entry by entry, rank-R form;
 *   oracle_bcss_pack         — the paper's m=2 element-order picture (Sec.
 *                              3.3) at b=1, block counts of Tbl. 1, Fig. 2's
 *                              storage ratios;
 *   oracle_bcss_flops        — the closed form of Tbl. 4 (MinCosts) and the
 *                              exact b=1 identity derived from Sec. 6.5.
 * tests/test_oracle_mutations.py plants single mistakes in a copy of this
 * file and checks that these pins fail on each.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int64_t ipow(int64_t base, int e)
{
    int64_t r = 1;
    for (int a = 0; a < e; ++a) r *= base;
    return r;
}

/*
 * Eq. (cob), elementwise definition (Sec. 2.5; the naive algorithm of
 * Fig. 1, left): gamma_{j_0..j_{m-1}} = sum over all (i_0..i_{m-1}) in
 * [0,n)^m of alpha_{i} * prod_k chi_{j_k, i_k}.  Every one of the p^m
 * entries of C is computed independently; nothing exploits symmetry.
 */
void oracle_sttsm_bruteforce(int m, int64_t n, int64_t p, const double* A, const double* X, double* C)
{
    int64_t nm = ipow(n, m), pm = ipow(p, m);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t jl = 0; jl < pm; ++jl) {
        int64_t j[16];
        int64_t r = jl;
        for (int k = 0; k < m; ++k) { j[k] = r % p; r /= p; }
        double acc = 0.0;
        for (int64_t il = 0; il < nm; ++il) {
            int64_t s = il;
            double prod = A[il];
            for (int k = 0; k < m; ++k) {
                int64_t ik = s % n;
                s /= n;
                prod *= X[j[k] + ik * p];
            }
            acc += prod;
        }
        C[jl] = acc;
    }
}

/*
 * Mode-k product (App. A): C = A x_k B with
 *   C_{i_0..i_{k-1} j i_{k+1}..} = sum_{i_k} A_{i_0..i_{m-1}} beta_{j, i_k},
 * written here as plain loops (no permutation, no BLAS).  dims[] holds the
 * extent of every mode of the input; B is q x dims[k], column-major.
 */
static void mode_k_product(int m, const int64_t* dims, int k, const double* in, int64_t q, const double* B, double* out)
{
    int64_t left = 1, right = 1;
    for (int a = 0; a < k; ++a) left *= dims[a];
    for (int a = k + 1; a < m; ++a) right *= dims[a];
    int64_t nk = dims[k];
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t r = 0; r < right; ++r) {
        for (int64_t j = 0; j < q; ++j) {
            double* o = out + left * (j + q * r);
            for (int64_t l = 0; l < left; ++l) o[l] = 0.0;
            for (int64_t i = 0; i < nk; ++i) {
                const double* src = in + left * (i + nk * r);
                double bji = B[j + i * q];
                for (int64_t l = 0; l < left; ++l) o[l] += src[l] * bji;
            }
        }
    }
}

/*
 * Successive mode products (Fig. 1, right; the temporaries T^(m-1), ...,
 * T^(1) of Sec. 5.2): out = A x_{m-1} X_{m-1} x_{m-2} ... x_0 X_0, applied
 * from the last mode to the first as the paper's loops do.  X_k is
 * q[k] x n, column-major.  With every X_k = X this is [A; X, ..., X].
 * No symmetry is exploited.  Returns 0, or -1 if a temporary cannot be
 * allocated.
 */
int oracle_ttm_chain(int m, int64_t n, const double* A, const int64_t* q, const double* const* Xs, double* out)
{
    int64_t dims[16];
    for (int a = 0; a < m; ++a) dims[a] = n;
    int64_t cur_size = ipow(n, m);
    const double* cur = A;
    double* owned = NULL;
    for (int k = m - 1; k >= 0; --k) {
        int64_t next_size = cur_size / dims[k] * q[k];
        double* next = (k == 0) ? out : (double*)malloc(sizeof(double) * (size_t)next_size);
        if (!next) { free(owned); return -1; }
        mode_k_product(m, dims, k, cur, q[k], Xs[k], next);
        free(owned);
        owned = (k == 0) ? NULL : next;
        cur = next;
        dims[k] = q[k];
        cur_size = next_size;
    }
    return 0;
}

/*
 * Selected entries of C (Sec. 4.1, written for one entry):
 *   gamma_j = A x_{m-1} x_{j_{m-1}} x_{m-2} ... x_0 x_{j_0},
 * i.e. m vector contractions, last mode first.  J holds count tuples of m
 * indices (row-major).  Returns 0, or -1 if a temporary cannot be allocated.
 */
int oracle_sttsm_entries(int m, int64_t n, int64_t p, const double* A, const double* X, const int64_t* J, int64_t count, double* out)
{
    int64_t tmp_len = ipow(n, m - 1);
    int fail = 0;
#pragma omp parallel
    {
        double* v0 = (double*)malloc(sizeof(double) * (size_t)(tmp_len > 0 ? tmp_len : 1));
        double* v1 = (double*)malloc(sizeof(double) * (size_t)(tmp_len > 0 ? tmp_len : 1));
        if (!v0 || !v1) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < count; ++t) {
            if (!v0 || !v1) continue;
            const int64_t* j = J + (int64_t)m * t;
            const double* cur = A;
            int64_t len = ipow(n, m);
            double* bufs[2] = {v0, v1};
            int which = 0;
            for (int k = m - 1; k >= 0; --k) {
                int64_t inner = len / n;
                double* nxt = bufs[which];
                for (int64_t l = 0; l < inner; ++l) nxt[l] = 0.0;
                for (int64_t i = 0; i < n; ++i) {
                    double x = X[j[k] + i * p];
                    const double* src = cur + inner * i;
                    for (int64_t l = 0; l < inner; ++l) nxt[l] += src[l] * x;
                }
                cur = nxt;
                len = inner;
                which ^= 1;
            }
            out[t] = cur[0];
        }
        free(v0);
        free(v1);
    }
    return fail ? -1 : 0;
}

/*
 * Next non-decreasing tuple over [0, nbar) in the order of the nested loops
 * "for t_{m-1} = 0..nbar-1, for t_{m-2} = 0..t_{m-1}, ..., for t_0 = 0..t_1"
 * (the loop structure of Figs. 2-4 and Fig. 1).  Returns 0 after the last.
 */
static int next_sorted_tuple(int m, int64_t nbar, int64_t* t)
{
    for (int a = 0; a < m; ++a) {
        int64_t upper = (a + 1 < m) ? t[a + 1] : nbar - 1;
        if (t[a] < upper) {
            ++t[a];
            for (int c = 0; c < a; ++c) t[c] = 0;
            return 1;
        }
    }
    return 0;
}

/* Number of stored blocks of BCSS, counted by walking the upper
 * hypertriangle (Sec. 4.3, 5.3). */
int64_t oracle_bcss_count_blocks(int m, int64_t nbar)
{
    if (nbar <= 0) return 0;
    int64_t t[16] = {0};
    int64_t count = 1;
    while (next_sorted_tuple(m, nbar, t)) ++count;
    return count;
}

/*
 * BCSS (Sec. 3.3, 4.3, 5.3): A is cut into b^m blocks; only blocks whose
 * block indices satisfy ibar_0 <= ... <= ibar_{m-1} are stored.  Stored
 * blocks follow the nested-loop order of the paper's algorithms (last block
 * index outermost), which for m = 2, b = 1 is the element order pictured in
 * Sec. 3.3.  Each block is a dense b^m array in dimensional order (App. A).
 * Entries of a block that fall beyond n (when b does not divide n; nbar =
 * ceil(n/b), App. B) are zero.
 */
void oracle_bcss_pack(int m, int64_t n, int b, const double* dense, double* out)
{
    int64_t nbar = (n + b - 1) / b;
    int64_t bm = ipow(b, m);
    int64_t t[16] = {0};
    int64_t blk = 0;
    do {
        double* dst = out + blk * bm;
        for (int64_t e = 0; e < bm; ++e) {
            int64_t r = e, off = 0, stride = 1;
            int inside = 1;
            for (int a = 0; a < m; ++a) {
                int64_t i = t[a] * b + r % b;
                r /= b;
                if (i >= n) inside = 0;
                off += i * stride;
                stride *= n;
            }
            dst[e] = inside ? dense[off] : 0.0;
        }
        ++blk;
    } while (next_sorted_tuple(m, nbar, t));
}

/*
 * Flop count of the algorithm-by-blocks of Fig. 5 (mD) when the partial
 * symmetry of every temporary is exploited (Thm. 1, Sec. 6.3), counted by
 * walking the loops: at level d (d = 0..m-1, producing T^(m-1-d), T^(0) = C)
 * every node is a non-decreasing (d+1)-tuple of C-block indices over
 * [0, pbar); every node computes the unique blocks of its temporary, one per
 * non-decreasing (m-1-d)-tuple over [0, nbar); every such block sums nbar
 * contributions, each a b_C x b_A block of X applied to one mode of a block
 * with b_A^{m-d} b_C^d entries, i.e. 2 b_C^{d+1} b_A^{m-d} flops.
 */
double oracle_bcss_flops(int m, int64_t n, int64_t p, int bA, int bC)
{
    int64_t nbar = (n + bA - 1) / bA, pbar = (p + bC - 1) / bC;
    double total = 0.0;
    for (int d = 0; d < m; ++d) {
        int64_t nodes = oracle_bcss_count_blocks(d + 1, pbar);
        int64_t out_blocks = (m - 1 - d == 0) ? 1 : oracle_bcss_count_blocks(m - 1 - d, nbar);
        double per = 2.0 * (double)ipow(bC, d + 1) * (double)ipow(bA, m - d);
        total += (double)nodes * (double)out_blocks * (double)nbar * per;
    }
    return total;
}
