// plan.h — host-side plans of the algorithm-by-blocks (Fig. 5 with Thm. 1):
// per level, the parent nodes, the unique output blocks, the gather table G
// and the tile list; cached per shape in library-owned device memory.
#pragma once

#include <stdint.h>
#include <vector>
#include "common.cuh"
#include "sttsm.h"

namespace sttsm {

// BF16 pieces of a precision (0 for FP64), whether its last level sums in
// FP64 (the R64 precisions), and whether the library accepts it.
inline int prec_npiece(int prec)
{
    return (prec == STTSM_BF16X6 || prec == STTSM_BF16X6_R64) ? 3 : (prec == STTSM_BF16X3 || prec == STTSM_BF16X3_R64) ? 2 : 0;
}
inline bool prec_r64(int prec) { return prec == STTSM_BF16X6_R64 || prec == STTSM_BF16X3_R64; }
inline bool prec_valid(int prec) { return prec == STTSM_FP64 || prec_npiece(prec) > 0; }
// Widest tile of the last level under the R64 precisions (32 FP64 sums per epilogue thread).
constexpr int R64_BN = 128;

struct LevelShape {
    int d, k;                  // level d writes T^(k), k = m-1-d
    int64_t nodes_parent;      // C(pbar+d-1, d) parent nodes (1 at level 0)
    int64_t nodes_out;         // C(pbar+d, d+1) child nodes
    int64_t P_parent;          // unique blocks per parent node: C(nbar+k, k+1)
    int64_t P_out;             // unique blocks per child node: C(nbar+k-1, k) (1 if k = 0)
};

// Shape facts of one sttsm instance (host only, no allocation).
struct Shape {
    int m, b;
    int64_t n, p, nbar, pbar;
    int64_t bm;                // b^m
    int64_t R;                 // b^(m-1)
    LevelShape lv[STTSM_MAX_M];
    int64_t buf_elems[2];      // ping-pong temporaries (elements)
};

// Returns 0 and fills s, or an sttsm_status for unsupported sizes.
int make_shape(int m, int64_t n, int64_t p, int b, Shape* s);

// Split-precision launches of a shape whose contraction n̄ b is at most 64
// use the small-tile kernel (128 x 64 tiles).
inline bool tc_small_mode(const Shape& s) { return s.nbar * s.b <= 64; }

// Split-precision shapes whose block size is a multiple of 16 and whose
// output blocks hold a multiple of 128 rows take the TMA-fed kernel
// (temporaries stored as BF16 pieces).
inline bool tc_tma_mode(const Shape& s) { return !tc_small_mode(s) && s.b % 16 == 0 && s.R % 128 == 0; }
// TMA-fed block sizes other than 32, 64 and multiples of 128 load one box per
// 16-wide K slice (32-byte swizzle, 16-row atoms) instead of one per 32-wide
// stage (64-byte swizzle, 32-row atoms): every b^q is then a multiple of the
// atom height.
inline bool tma_sw32_b(int b) { return !(b == 32 || b == 64 || b % 128 == 0); }
inline bool tma_sw32(const Shape& s) { return tma_sw32_b(s.b); }

// TMA-fed levels whose 128-row tiles are 16 values of the fastest row index
// times 8 of the next (Tile::pad0 = 1): the 16-wide slice form (b = 48, 80,
// 112, ...) with m <= 4, at levels where some insertion position q >= 1 has
// runs of b^q rows that neither divide 128 nor are multiples of it.  Every A
// box of such a tile is one TMA load whatever q is.
bool tma_order16x8(const Shape& s, int d);

// Host tile list and G table of level d (appended to the given vectors).
// Tiles cover, for every parent node, P_out * R rows in steps of BM and the
// parent's children * b columns in steps of BN; with order16x8 (BM = 128) a
// tile's rows are row0 + (t mod 16) + b (t div 16), t < 128, instead of
// row0 + t.
void build_level_tiles(const Shape& s, int d, int BM, int BN, int32_t inst, std::vector<Tile>& tiles,
                       bool order16x8 = false);
// Tiles of level d in the in-block-symmetry mode (sym.cuh): for every parent
// node its canonical rows rho in steps of BM times the parent's children * b
// columns in steps of BN; pad0 = SYM_TILE | tie pattern << 8 | u_0 << 16,
// pad1 = the parent's canonical rows.  For short-contraction shapes of order
// m <= 5 only (nbar b <= 64, pbar < 65536: sym_shape_ok).
bool sym_shape_ok(const Shape& s);
void build_level_tiles_sym(const Shape& s, int d, int BM, int BN, int32_t inst, std::vector<Tile>& tiles);
// Number of tiles build_level_tiles emits for level d (counted, not built).
int64_t level_tile_count(const Shape& s, int d, int BM, int BN);
// G table of level d ([P_out][nbar]) followed by its offset table OFF
// ([k+1][R]); level_G_size is the length of the G part.
void build_level_G(const Shape& s, int d, std::vector<int32_t>& G);
inline int64_t level_G_size(const Shape& s, int d) { return s.lv[d].P_out * s.nbar; }

// The last two levels fused (kernels_pair.cu): FP32 short contractions whose
// contraction and output widths are at most 64 (nbar b <= 64, pbar b <= 64),
// m >= 2, and whose unit of work (G_s trailing index tuples, Kc G_s <= 128
// level m-2 rows with Kc = nbar b rounded up to 4) keeps its T^(1) slice of
// Kc x pbar x (b G_s rounded up to 4) entries within PAIR_U_MAX.
constexpr int PAIR_U_MAX = 10240;
constexpr int PAIR_ROWS = 128;
int pair_group(const Shape& s);          // G_s of the fused units
bool pair_mode(const Shape& s);
// Units of the fused launch (fields as kernels_pair.cu reads them), appended.
void build_pair_tiles(const Shape& s, int32_t inst, std::vector<Tile>& tiles);

struct DevPlan {
    Shape shape;
    int BM, BN;
    int ntiles[STTSM_MAX_M];
    int maxcols[STTSM_MAX_M];   // widest tile of each level
    Tile* d_tiles[STTSM_MAX_M];
    int32_t* d_G[STTSM_MAX_M];
    Tile* d_pair;               // fused last two levels (pair_mode shapes of the split plans), else nullptr
    int npair;
};

// Cached device plan for (shape, tile sizes) on the current device; nullptr
// on allocation failure.  Thread-safe.  The first call for a shape allocates
// and copies synchronously (do it before any stream capture).  bn_last (0 =
// BN): tile width bound of the last level.
// sym: level tiles in the in-block-symmetry mode (build_level_tiles_sym).
const DevPlan* get_dev_plan(int m, int64_t n, int64_t p, int b, int BM, int BN, int bn_last = 0, bool sym = false);

}  // namespace sttsm
