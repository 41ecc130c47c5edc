// common.cuh — shared definitions of the sttsm library (host + device).
//
// BCSS indexing (Sec. 3.3, 4.3, 5.3 of Schatz/Low/van de Geijn/Kolda, arXiv
// 1301.7744): a stored block is identified by a non-decreasing tuple of
// block indices; its storage position is the colex rank
//     rank(s_0 <= ... <= s_{k-1}) = sum_t C(s_t + t, t + 1),
// which enumerates the tuples in the order of the paper's nested loops
// (last index slowest).
#pragma once

#include <stdint.h>
#include <cuda_runtime.h>

#define STTSM_HD __host__ __device__ __forceinline__

constexpr int STTSM_MAX_M = 8;

// C(x, y) for 0 <= y <= 8; 0 when x < y.  Exact for every value used here.
STTSM_HD int64_t binom_small(int64_t x, int y)
{
    if (y < 0 || x < y) return 0;
    int64_t c = 1;
    for (int i = 1; i <= y; ++i) c = c * (x - y + i) / i;
    return c;
}

// Colex rank of a sorted tuple.
STTSM_HD int64_t colex_rank(const int32_t* s, int k)
{
    int64_t r = 0;
    for (int t = 0; t < k; ++t) r += binom_small((int64_t)s[t] + t, t + 1);
    return r;
}

// Inverse of colex_rank for tuples of length k.
STTSM_HD void colex_unrank(int64_t r, int k, int32_t* s)
{
    for (int t = k - 1; t >= 0; --t) {
        // largest v with C(v + t, t + 1) <= r; C(v + t, t + 1) grows with v
        int64_t lo = 0, hi = 1;
        while (binom_small(hi + t, t + 1) <= r) hi *= 2;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            if (binom_small(mid + t, t + 1) <= r) lo = mid; else hi = mid;
        }
        s[t] = (int32_t)lo;
        r -= binom_small(lo + t, t + 1);
    }
}

// One unit of work of a level launch: an M-tile of output rows of one parent
// node times a range of output columns (children j-blocks x b).
struct Tile {
    int32_t inst;        // instance descriptor index (batched launches)
    int32_t parent;      // rank of the parent node among level d-1 nodes (0 at level 0)
    int32_t child_base;  // rank of the parent's first child among level d nodes
    int32_t row0;        // first output row of the tile within the parent's rows (see pad0)
    int32_t col0;        // first output column (j index, = jbar * b + c)
    int32_t ncols;       // valid columns in this tile
    int32_t pad0, pad1;  // TMA-fed tiles: pad0 = 1 when the rows are 16 fastest x 8 next (plan.h)
};

// Everything a level kernel needs to know about one sttsm instance at one
// level d (k = m-1-d: the level reads T^(k+1) and writes T^(k); T^(m) = A,
// T^(0) = C).  Offsets are in elements.
struct LevelInst {
    const void* parent;     // T^(k+1) storage: [parent node][stored block][b^m]
    void* out;              // T^(k) storage:   [child node][stored block][b^m]
    const int32_t* G;       // [P_out][nbar]: (rank of sort(prefix + ibar)) << 3 | insertion position q
    const int32_t* OFF;     // [k+1][R]: off_q(rr) (below); OFF[k][rr] is also the output row offset
    const void* X;          // FP64 path: X (p x n column-major); split path: unused
    int32_t m, b, k, nbar;
    int32_t n, p;           // unpadded sizes (bounds of X)
    int32_t R;              // rows per output block = b^(m-1)
    int32_t Ktot;           // nbar * b
    int64_t bm;             // b^m
    int64_t P_parent;       // stored blocks per parent node
    int64_t P_out;          // stored blocks per child node
    int64_t rows_per_parent;  // P_out * R
    int32_t bpow[STTSM_MAX_M + 1];
    int32_t out_np;         // 0: FP32 output; else BF16 pieces per block [node][block][piece][b^m]
    int32_t order16x8;      // TMA-fed tiles: rows row0 + (t mod 16) + b (t div 16) (see plan.h)
    int32_t sym_full;       // in-block-symmetry tiles (sym.cuh): 1 where out is the call's result
                            // (every entry written), 0 for a temporary (canonical entries only)
};

// Rows of a tile are mapped to (prefix block pr, row rr) by
//     g = row0 + t, pr = g / R, rr = g % R,
// and the gathered operand entry for contraction index kk = ibar * b + a is
//     parent[(parent_node * P_parent + rank) * b^m + off_q(rr) + a * b^q],
//     off_q(rr) = rr % b^q + b^(q+1) * (rr / b^q),
// (tabulated per level as OFF[q][rr], so kernels do no integer division per
// entry), where (rank, q) = G[pr][ibar]: the stored block of the sorted tuple and the
// local mode the contraction index occupies in it (inserting ibar before the
// first prefix entry >= ibar).  The output entry (rr, c) of child jbar goes to
//     out[(child_node * P_out + pr) * b^m + rr % b^k + b^k * c + b^(k+1) * (rr / b^k)],
// i.e. the new mode k lands between the k symmetric modes and the trailing
// modes, keeping every temporary in dimensional order.
