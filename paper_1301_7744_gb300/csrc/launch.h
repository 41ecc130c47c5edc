// launch.h — internal host-side launchers of the sttsm kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include "common.cuh"

namespace sttsm {

// Split-precision level launch: per-instance data plus the TMA descriptor of
// that instance's X pieces ([npiece][rows][Kp] BF16, K-major rows).
struct TcInst {   // CUtensorMap first: inherits its 64-byte alignment
    CUtensorMap tmX;
    LevelInst L;
};

int launch_bcss_pack(const void* dense, void* bcss, int m, int64_t n, int b, int dtype, cudaStream_t s);
int launch_bcss_unpack(const void* bcss, void* dense, int m, int64_t n, int b, int dtype, cudaStream_t s);
int launch_split_x(const float* X, void* out, int p, int n, int rows, int Kp, int npiece, cudaStream_t s);

// Batched X split: instance i owns CTAs [first_block, first_block + ceil(rows * Kp / 256)).
struct SplitDesc {
    const float* X;
    void* out;
    int p, n, rows, Kp;
    int64_t first_block;
};
int launch_split_x_batch(const SplitDesc* d_desc, int count, int blocks, int npiece, cudaStream_t s);
int launch_level_fp64(const LevelInst& inst0, const LevelInst* d_insts, const Tile* d_tiles, int ntiles,
                      int num_sms, cudaStream_t s);

// Tensor-core level launch (tcgen05, BF16 pieces, FP32 accumulation in TMEM).
// Tiles are 128 rows x up to TC_BN columns.  Either inst0 (single instance,
// d_insts == nullptr) or d_insts[tile.inst] describes each tile.
constexpr int TC_BM = 128;
constexpr int TC_BN = 256;
constexpr int TC_KC = 32;
int launch_level_tc(int npiece, const TcInst& inst0, const TcInst* d_insts, const Tile* d_tiles, int ntiles,
                    int num_sms, int* d_status, cudaStream_t s);
// The same with the register sums in FP64 (the R64 precisions); every tile at
// most 128 columns (max_cols: the widest).
int launch_level_tc_r64(int npiece, const TcInst& inst0, const TcInst* d_insts, const Tile* d_tiles, int ntiles,
                        int num_sms, int* d_status, int max_cols, cudaStream_t s);

// FP32 CUDA-core kernel for short contractions (n̄ b <= 64): tiles of 128 rows
// x <= 64 columns, X read from the instance's FP32 X (LevelInst::X).
// r64: instances at their last level (k = 0) add the FP32 sums of their
// contraction blocks in FP64 (the R64 precisions).  sym: some tiles were built
// by build_level_tiles_sym (Tile::pad0 = SYM_TILE: canonical entries only,
// sym.cuh; a launch may mix both kinds); 0 runs the kernel without that code.
int launch_level_small_f32(const LevelInst& inst0, const LevelInst* d_insts, const Tile* d_tiles, int ntiles,
                           int num_sms, cudaStream_t s, int r64 = 0, int sym = 0);
int launch_level_small_f32_tc(const TcInst* d_insts, const Tile* d_tiles, int ntiles, int num_sms, cudaStream_t s,
                              int r64 = 0, int sym = 0);

// Levels m-2 and m-1 of short contractions fused (kernels_pair.cu): the
// descriptor describes level m-2 with out = C; tiles from build_pair_tiles.
int launch_level_pair_f32(const LevelInst& inst0, const LevelInst* d_insts, const Tile* d_tiles, int ntiles,
                          int num_sms, cudaStream_t s);
int launch_level_pair_f32_tc(const TcInst* d_insts, const Tile* d_tiles, int ntiles, int num_sms, cudaStream_t s);
// Whether short contractions run their last two levels fused (sttsm_set_fused_tail):
// in single calls (mode >= 1), and in batch plans and serving (mode 2).
bool fused_tail_enabled();
bool fused_tail_in_batches();

// Whether split-precision levels of short-contraction shapes compute canonical
// entries only (sttsm_set_inblock_symmetry; sym.cuh): the switch is on, the
// FP32 short-contraction kernel runs them and the shape fits the tile
// encoding (sym_shape_ok).
bool inblock_sym_enabled();
struct Shape;
bool sym_levels(const Shape& s, int prec);

// Kernel for short contractions under the split precisions: 0 = FP32 CUDA-core
// kernel (default), 1 = tcgen05 small-tile kernel (sttsm_set_small_kernel).
int small_kernel_kind();

// Small-tile variant: every tile has a contraction of at most TC_SMALL_K
// (two stages) and at most TC_SMALL_BN columns; X maps with box rows 64.
constexpr int TC_SMALL_K = 64;
constexpr int TC_SMALL_BN = 64;
int launch_level_tc_small(int npiece, const TcInst& inst0, const TcInst* d_insts, const Tile* d_tiles, int ntiles,
                          int num_sms, int* d_status, cudaStream_t s);

// TMA-fed variant (kernels_tma.cu): parent temporaries (and A) as BF16 pieces
// [node][block][piece][b^m]; tmA[q] maps the parent for insertion position q.
constexpr int TMA_NX = 8;
struct TmaInst {
    CUtensorMap tmX[TMA_NX];       // X pieces with box rows 32 (i + 1); a tile of c columns loads 32 ceil(c / 32) rows
    CUtensorMap tmA[STTSM_MAX_M];
    LevelInst L;
};
// out_kind: TMA_OUT_PIECES writes the next level's operand as BF16 pieces,
// TMA_OUT_C writes FP32 C (the last level, k = 0: a row's columns contiguous),
// TMA_OUT_F32 writes FP32 at a level k >= 1 (the all-but-one result).
// sw32: every instance of the launch has b an odd multiple of 16 (one box per
// 16-wide K slice, 32-byte swizzle); otherwise every instance has b a multiple
// of 32 (one box per 32-wide stage).
// TMA_OUT_C64 writes C like TMA_OUT_C with the register sums in FP64 (the R64
// precisions; tiles of at most 128 columns).
constexpr int TMA_OUT_PIECES = 0, TMA_OUT_C = 1, TMA_OUT_F32 = 2, TMA_OUT_C64 = 3;

// A wait that never completes, bounded by limit_ns; raises *d_status on timeout.
int launch_wait_probe(int* d_status, unsigned long long limit_ns, cudaStream_t s);
// max_cols: the widest tile of the launch; launches of tiles <= 64 columns wide
// run with more, smaller pipeline stages.
int launch_level_tma(int npiece, const TmaInst& inst0, const TmaInst* d_insts, const Tile* d_tiles, int ntiles,
                     int num_sms, int* d_status, int out_kind, bool sw32, int max_cols, cudaStream_t s);
int launch_split_bcss(const float* in, void* out, int64_t nblocks, int64_t bm, int npiece, cudaStream_t s);

// Tensor maps of a BF16-piece parent array with nblocks stored blocks (all
// nodes) for insertion positions q = 0..k of a level (see kernels_tma.cu).
// order16x8: the level's tiles are 16 fastest x 8 next rows (plan.h tma_order16x8).
int make_a_tensor_maps(CUtensorMap* maps, const void* pieces, int64_t nblocks, int npiece, int b, int m, int k,
                       bool order16x8 = false);

// Builds the TMA descriptor of an X-piece array (box: TC_KC x box_rows x npiece).
int make_x_tensor_map(CUtensorMap* map, const void* xpieces, int npiece, int rows, int Kp, int box_rows = TC_BN);

}  // namespace sttsm
