// kernels_tma.cu — the split-precision level kernel with the A operand loaded by
// TMA from BF16 pieces (block sizes b that are multiples of 16 and whose output
// blocks hold a multiple of 128 rows).
//
// The operands are those of level_tc_kernel (kernels_tc.cu): rows of stored
// parent blocks gathered through G times X.  Here the parent temporaries (and A,
// pre-split once) are stored as BF16 pieces, [node][block][piece][b^m], so every
// 32-wide contraction stage of a 128-row tile is one box of one stored block
// when b is a multiple of 32 (64-byte swizzle); otherwise (b = 16, 48, 80, ...)
// each 16-wide MMA slice of the stage is a box of the stored block holding that
// slice (32-byte swizzle):
//   * insertion position q = 0: the contraction index is the block's fastest
//     mode, rows are b apart -> a 3-D K-major box {32 (16), 128, NP};
//   * q >= 1: rows are contiguous in runs of b^q and the contraction index is
//     b^q apart -> a 5-D MN-major box {32 (16) rows, 32 (16) k, atoms, outer, NP}
//     in 32-row (16-row) swizzle atoms; when b^q neither divides 128 nor is a
//     multiple of it (b^q = 48, 80, ...), the 16-row atoms of the tile are
//     loaded one by one, the pieces of an atom side by side,
// which is how the permutation of App. A (permute before dgemm) becomes a choice
// of tensor map and operand major-ness per stage instead of a data movement.
//
// CTA = 18 warps, one per SM, persistent over the tile list (launches whose
// tiles are all <= 64 columns: 10 warps with 8 epilogue warps, two CTAs per SM):
//   warps 0-15  epilogue: D0 partials (x0*y0, restarted every 128 contraction
//               indices of a tile) folded into FP32
//               registers, D1 (cross products) added at the end of the tile; the
//               row is written as BF16 pieces for the next level, FP32 into C at
//               the last level, or FP32 at level m-2 for the all-but-one result;
//   warp 16     TMEM allocation and the MMA-issuing thread;
//   warp 17     the TMA-issuing thread (A box per stage by q, X pieces box).
#include <cuda_bf16.h>
#include <cuda.h>
#include <mutex>
#include <type_traits>
#include "common.cuh"
#include "launch.h"
#include "tc_ptx.cuh"

namespace sttsm {

using namespace ptx;

namespace {

// D0 (x0*y0) restarts: the first group of a tile spans T_GS0 stages (room for
// the epilogue to finish the previous tile's stores before the first drain),
// the later ones T_GS stages.  Groups of 4 stages (128 contraction indices)
// halve the drains of groups of 2 on the m=3 n=768 b=64 step (+1.5 %) for a
// sampled error of 3.3e-7 instead of 2.4e-7; 8 stages gave 6.1e-7.
constexpr int T_GS = 4, T_GS0 = 4;
__host__ __device__ constexpr bool d0_group_start(int ks) { return ks == 0 || (ks >= T_GS0 && (ks - T_GS0) % T_GS == 0); }
__host__ __device__ constexpr bool d0_group_end(int ks, int nk)
{
    return ks == nk - 1 || ks == T_GS0 - 1 || (ks >= T_GS0 && (ks - T_GS0) % T_GS == T_GS - 1);
}
__host__ __device__ constexpr int d0_groups(int nk) { return nk <= T_GS0 ? 1 : 1 + (nk - T_GS0 + T_GS - 1) / T_GS; }

// A run of b^q contiguous rows (insertion position q >= 1) that neither holds
// whole 128-row tiles nor divides 128 (b^q = 48, 80, 112, 144, ...): the tile's
// 16-row atoms are loaded one by one.
__host__ __device__ constexpr bool atomwise_run(int bq) { return (bq % 128) != 0 && (128 % bq) != 0; }

template <int NP>
struct SmemT {
    static constexpr int A_PLANE = TC_BM * TC_KC * 2;
    static constexpr int B_PLANE = TC_BN * TC_KC * 2;
    static constexpr int STAGE = NP * (A_PLANE + B_PLANE);
    static constexpr int STAGES = NP == 3 ? 3 : 4;
    // launches whose tiles are all <= 64 columns: X planes of 64 rows, more stages
    static constexpr int NSTAGE = NP * (A_PLANE + B_PLANE / 4);
    static constexpr int NSTAGES = STAGES * STAGE / NSTAGE;
    static constexpr int MAXST = NSTAGES > STAGES ? NSTAGES : STAGES;
    static constexpr int BYTES = STAGES * STAGE + 1024 + 256;
    // the two-CTAs-per-SM form for launches of tiles <= 64 columns (8 epilogue warps)
    static constexpr int NSTAGES_P = NP == 3 ? 3 : 4;
    static constexpr int BYTES_P = NSTAGES_P * NSTAGE + 1024 + 256;
};

// acc[0..63] += 64 consecutive TMEM columns of this warp's lanes from taddr
__device__ __forceinline__ void tmem_fold64(float* acc, uint32_t taddr)
{
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float v[8];
        tmem_ld_32x32b_x8(taddr + c * 8, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[c * 8 + i] += v[i];
    }
}

// acc[0..n) += n consecutive TMEM columns (n a multiple of 8, < MAXC)
template <int MAXC = 64>
__device__ __forceinline__ void tmem_fold_n(float* acc, uint32_t taddr, int n)
{
#pragma unroll
    for (int c = 0; c < MAXC / 8; ++c) {
        if (c * 8 >= n) break;
        float v[8];
        tmem_ld_32x32b_x8(taddr + c * 8, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[c * 8 + i] += v[i];
    }
}

// acc[0..31] += 32 consecutive TMEM columns, accumulated in FP64 (the C-block
// reduction of the R64 precisions)
__device__ __forceinline__ void tmem_fold32_f64(double* acc, uint32_t taddr)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float v[8];
        tmem_ld_32x32b_x8(taddr + c * 8, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[c * 8 + i] += (double)v[i];
    }
}

}  // namespace

// EW epilogue warps: 16 (one CTA per SM, all 512 TMEM columns, tiles up to 256
// columns), or 8 for launches whose tiles are all <= 64 columns (two CTAs per
// SM, 128 TMEM columns and three or four narrow stages each, so twice as many
// tiles are in flight)
template <int NP, int OUT, bool SW32, int EW>
__global__ void __launch_bounds__((EW + 2) * 32, EW == 16 ? 1 : 2)
level_tma_kernel(const __grid_constant__ TmaInst inst0, const TmaInst* __restrict__ insts,
                 const Tile* __restrict__ tiles, int ntiles, int* status, int narrow)
{
    using S = SmemT<NP>;
    constexpr int MAXST = S::MAXST;
    constexpr int EPIW = EW, MMAW = EW, TMAW = EW + 1;
    constexpr uint32_t TCOLS = EW == 16 ? 512u : 128u;
    constexpr uint32_t D0OFF = EW == 16 ? (uint32_t)TC_BN : 64u;
    const int STAGES = EW == 16 ? (narrow ? S::NSTAGES : S::STAGES) : S::NSTAGES_P;
    const int STAGE_BYTES = (narrow || EW != 16) ? S::NSTAGE : S::STAGE;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + (EW == 16 ? S::STAGES * S::STAGE : S::NSTAGES_P * S::NSTAGE));
    uint32_t* tmem_holder = (uint32_t*)(bars + 2 * MAXST + 4);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (MAXST + s); };
    const uint32_t d0_full = bar0 + 8u * (2 * MAXST);
    const uint32_t d0_empty = bar0 + 8u * (2 * MAXST + 1);
    const uint32_t d1_empty = bar0 + 8u * (2 * MAXST + 2);
    const uint32_t drain_bar = bar0 + 8u * (2 * MAXST + 3);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(full_bar(s), 1); mbar_init(empty_bar(s), 1); }
        mbar_init(d0_full, 1);
        mbar_init(d0_empty, EPIW);
        mbar_init(d1_empty, EPIW);
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == MMAW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_holder)), "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    const uint32_t tmem_d1 = tmem_base;
    const uint32_t tmem_d0 = tmem_base + D0OFF;

    if (warp == TMAW) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_stage = -1;
            uint32_t last_phase = 0;
            bool ok = true;
            for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
                const Tile t = tiles[ti];
                if (narrow && t.ncols > 64) {   // a stage has room for 64 X rows only
                    *abort_flag = 1;
                    atomicExch(status, 1);
                    ok = false;
                    break;
                }
                const TmaInst& TI = insts ? insts[t.inst] : inst0;
                const LevelInst& I = TI.L;
                const int pr = t.row0 / I.R, rr0 = t.row0 - pr * I.R;
                const int32_t* Grow = I.G + (int64_t)pr * I.nbar;
                const int nk = (I.Ktot + TC_KC - 1) / TC_KC;
                // 16-wide slices: running (stored block, offset in it) and the insertion
                // positions whose runs are loaded atom by atom
                int sl_ib = 0, sl_a = 0;
                uint32_t amask = 0;
                const bool o16 = SW32 && I.order16x8;   // tile rows: 16 fastest x 8 next (one box per slice)
                if (SW32 && !o16)
                    for (int q = 1; q <= I.k; ++q) amask |= atomwise_run(I.bpow[q]) ? (1u << q) : 0u;
                const int o_f0 = rr0 % I.b, o_s0 = rr0 / I.b;
                for (int ks = 0; ks < nk; ++ks) {
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, status)) { ok = false; break; }
                    const int k0 = ks * TC_KC;
                    const uint32_t sA = smem_u32(smem + stage * STAGE_BYTES);
                    const uint32_t sB = sA + NP * S::A_PLANE;
                    // X box rows: the tile's columns rounded up to 32
                    const int xsel = (t.ncols + 31) / 32 - 1;
                    const uint32_t x_bytes = (uint32_t)(NP * (xsel + 1) * 32 * TC_KC * 2);
                    if (SW32) {
                        // one box per 16-wide K slice, each from the stored block
                        // holding that slice (the second slice is absent when the
                        // contraction ends inside the stage)
                        const int nsl = k0 + 16 < I.Ktot ? 2 : 1;
                        mbar_arrive_expect_tx(full_bar(stage), (uint32_t)(nsl * NP * (S::A_PLANE / 2)) + x_bytes);
                        for (int h = 0; h < nsl; ++h) {
                            const int ib = sl_ib, a0 = sl_a;
                            sl_a += 16;
                            if (sl_a == I.b) { sl_a = 0; ++sl_ib; }
                            const int32_t gq = __ldg(Grow + ib);
                            const int q = gq & 7;
                            const int bp = (int)(((int64_t)t.parent * I.P_parent + (gq >> 3)) * NP);
                            const uint32_t dA = sA + (uint32_t)(h * NP * (S::A_PLANE / 2));
                            if (o16) {
                                // {a, f, r1, r2, block x piece} at q = 0, {f, a, r1, r2, ...} at q >= 1
                                const int r1 = o_s0 % I.b, r2 = o_s0 / I.b;
                                if (q == 0) tma_load_5d(dA, &TI.tmA[0], a0, o_f0, r1, r2, bp, full_bar(stage));
                                else tma_load_5d(dA, &TI.tmA[q], o_f0, a0, r1, r2, bp, full_bar(stage));
                            } else if (q == 0) {
                                tma_load_3d(dA, &TI.tmA[0], a0, rr0, bp, full_bar(stage));
                            } else {
                                const int bq = I.bpow[q];
                                if ((amask >> q) & 1u) {
                                    // 16-row atoms one by one (each lies inside one run of
                                    // b^q contiguous rows), all pieces of an atom together
#pragma unroll 1
                                    for (int a = 0; a < TC_BM / 16; ++a) {
                                        const int r = rr0 + 16 * a;
                                        tma_load_5d(dA + (uint32_t)(a * NP * 512), &TI.tmA[q], 0, a0, (r % bq) >> 4, r / bq,
                                                    bp, full_bar(stage));
                                    }
                                } else {
                                    tma_load_5d(dA, &TI.tmA[q], 0, a0, (rr0 % bq) >> 4, rr0 / bq, bp, full_bar(stage));
                                }
                            }
                        }
                    } else {
                        const int ib = k0 / I.b, a0 = k0 - ib * I.b;
                        const int32_t gq = __ldg(Grow + ib);
                        const int q = gq & 7;
                        const int bp = (int)(((int64_t)t.parent * I.P_parent + (gq >> 3)) * NP);
                        mbar_arrive_expect_tx(full_bar(stage), (uint32_t)(NP * S::A_PLANE) + x_bytes);
                        if (q == 0) {
                            tma_load_3d(sA, &TI.tmA[0], a0, rr0, bp, full_bar(stage));
                        } else {
                            const int bq = I.bpow[q];
                            tma_load_5d(sA, &TI.tmA[q], 0, a0, (rr0 % bq) >> 5, rr0 / bq, bp, full_bar(stage));
                        }
                    }
                    tma_load_3d(sB, &TI.tmX[xsel], k0, t.col0, 0, full_bar(stage));
                    last_stage = stage;
                    last_phase = phase;
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok && last_stage >= 0) {
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(full_bar(last_stage), last_phase))
                    if (globaltimer() - t0 > WAIT_LIMIT_NS) break;
            }
        }
        __syncwarp();
    } else if (warp == MMAW) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, group_phase = 0, tile_phase = 0;
            bool ok = true, issued = false;
            for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
                const Tile t = tiles[ti];
                const TmaInst& TI = insts ? insts[t.inst] : inst0;
                const LevelInst& I = TI.L;
                const int pr = t.row0 / I.R;
                const int32_t* Grow = I.G + (int64_t)pr * I.nbar;
                const int nk = (I.Ktot + TC_KC - 1) / TC_KC;
                const int nmma = (t.ncols + 15) & ~15;
                const uint32_t idesc_k = idesc_bf16(nmma), idesc_mn = idesc_bf16_amn(nmma);
                // B piece planes are as tall as the X box the producer used
                const uint32_t b_plane = (uint32_t)(((t.ncols + 31) / 32) * 32 * TC_KC * 2);
                if (!mbar_wait(d1_empty, tile_phase ^ 1u, abort_flag, status)) { ok = false; break; }
                tile_phase ^= 1u;
                tc_fence_after();
                int sl_ib = 0, sl_a = 0;
                uint32_t amask = 0;
                if (SW32 && !I.order16x8)
                    for (int q = 1; q <= I.k; ++q) amask |= atomwise_run(I.bpow[q]) ? (1u << q) : 0u;
                for (int ks = 0; ks < nk; ++ks) {
                    // A major-ness, atom layout and presence of the two 16-wide K slices
                    bool mnk[2], valid[2], atom[2];
                    if (SW32) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            valid[h] = ks * TC_KC + 16 * h < I.Ktot;
                            const int q = valid[h] ? (__ldg(Grow + sl_ib) & 7) : 0;
                            mnk[h] = q != 0;
                            atom[h] = ((amask >> q) & 1u) != 0;
                            sl_a += 16;
                            if (sl_a == I.b) { sl_a = 0; ++sl_ib; }
                        }
                    } else {
                        const int ib = (ks * TC_KC) / I.b;
                        mnk[0] = mnk[1] = (__ldg(Grow + ib) & 7) != 0;
                        valid[0] = valid[1] = true;
                        atom[0] = atom[1] = false;
                    }
                    if (!mbar_wait(full_bar(stage), phase, abort_flag, status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sA = smem_u32(smem + stage * STAGE_BYTES);
                    const uint32_t sB = sA + NP * S::A_PLANE;
                    auto adesc = [&](int s, int kh) {
                        if (SW32) {
                            if (atom[kh])
                                return smem_desc_sw32_mn_lbo(sA + (uint32_t)(kh * NP * (S::A_PLANE / 2) + s * 512),
                                                             (uint32_t)(NP * 512));
                            const uint32_t a = sA + (uint32_t)((kh * NP + s) * (S::A_PLANE / 2));
                            return mnk[kh] ? smem_desc_sw32_mn(a) : smem_desc_sw32(a);
                        }
                        return mnk[kh] ? smem_desc_sw64_mn(sA + s * S::A_PLANE + kh * 1024)
                                       : smem_desc_sw64(sA + s * S::A_PLANE + kh * 32);
                    };
#pragma unroll
                    for (int kh = 0; kh < TC_KC / 16; ++kh) {
                        if (!valid[kh]) continue;
                        const uint32_t idesc = mnk[kh] ? idesc_mn : idesc_k;
#pragma unroll
                        for (int s = 0; s < NP; ++s) {
#pragma unroll
                            for (int u = 0; u < NP; ++u) {
                                if (s + u > NP - 1 || s + u == 0) continue;
                                const uint64_t bd = smem_desc_sw64(sB + u * b_plane + kh * 32);
                                const bool first = ks == 0 && kh == 0 && s == 0 && u == 1;
                                tc_mma(tmem_d1, adesc(s, kh), bd, idesc, first ? 0u : 1u);
                                issued = true;
                            }
                        }
                    }
                    const bool group_start = d0_group_start(ks);
                    if (group_start) {
                        if (!mbar_wait(d0_empty, group_phase ^ 1u, abort_flag, status)) { ok = false; break; }
                        group_phase ^= 1u;
                        tc_fence_after();
                    }
#pragma unroll
                    for (int kh = 0; kh < TC_KC / 16; ++kh)
                        if (valid[kh])
                            tc_mma(tmem_d0, adesc(0, kh), smem_desc_sw64(sB + kh * 32), mnk[kh] ? idesc_mn : idesc_k,
                                   (group_start && kh == 0) ? 0u : 1u);
                    tc_commit(empty_bar(stage));
                    if (d0_group_end(ks, nk)) tc_commit(d0_full);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok && issued) {
                tc_commit(drain_bar);
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(drain_bar, 0))
                    if (globaltimer() - t0 > WAIT_LIMIT_NS) break;
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue (warps 0-15)
        // warp (quad, cq) owns TMEM lanes 32 quad.. (rows) and the cq-th quarter
        // of the tile's columns (a multiple of 8, <= 64), so narrow tiles keep
        // all 16 warps busy.  The fold reads the quarter's own columns (all 64
        // of a full quarter with a fixed-length loop).
        const int quad = warp & 3, cq = warp >> 2;
        const int row = quad * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        uint32_t group_phase = 0;
        bool ok = true;
        // FP32 register sums, or FP64 ones for C under the R64 precisions (32 columns
        // per thread: tiles of at most 128 columns)
        constexpr bool R64 = OUT == TMA_OUT_C64;
        constexpr int AW = (R64 || EW != 16) ? 32 : 64;
        constexpr int PARTS = EW / 4;               // column parts of a tile (4 or 2)
        using AccT = typename std::conditional<R64, double, float>::type;
        AccT acc[AW];
        for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
            const Tile t = tiles[ti];
            const TmaInst& TI = insts ? insts[t.inst] : inst0;
            const LevelInst& I = TI.L;
            const int nk = (I.Ktot + TC_KC - 1) / TC_KC;
            const int ngroups = d0_groups(nk);
            // (the FP32 writer of C keeps whole 64-column quarters: its rows are
            // contiguous, and longer runs per thread store faster)
            const int cw = R64 ? 32 : OUT == TMA_OUT_C ? AW : ((((t.ncols + 15) & ~15) + PARTS - 1) / PARTS + 7) & ~7;
            const int colbase = cq * cw;
            const bool active = colbase < t.ncols;
#pragma unroll
            for (int i = 0; i < AW; ++i) acc[i] = 0;
            for (int gi = 0; gi < ngroups; ++gi) {
                if (!mbar_wait(d0_full, group_phase, abort_flag, status)) { ok = false; break; }
                group_phase ^= 1u;
                tc_fence_after();
                if (active) {
                    if constexpr (R64) tmem_fold32_f64(acc, tmem_d0 + lane_off + (uint32_t)colbase);
                    else if constexpr (AW == 64) {
                        if (cw == 64) tmem_fold64(acc, tmem_d0 + lane_off + (uint32_t)colbase);
                        else tmem_fold_n<64>(acc, tmem_d0 + lane_off + (uint32_t)colbase, cw);
                    } else tmem_fold_n<AW + 8>(acc, tmem_d0 + lane_off + (uint32_t)colbase, cw);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(d0_empty);
            }
            if (!ok) break;
            if (active) {
                if constexpr (R64) tmem_fold32_f64(acc, tmem_d1 + lane_off + (uint32_t)colbase);
                else if constexpr (AW == 64) {
                    if (cw == 64) tmem_fold64(acc, tmem_d1 + lane_off + (uint32_t)colbase);
                    else tmem_fold_n<64>(acc, tmem_d1 + lane_off + (uint32_t)colbase, cw);
                } else tmem_fold_n<AW + 8>(acc, tmem_d1 + lane_off + (uint32_t)colbase, cw);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(d1_empty);
            const int g = t.row0 + (SW32 && I.order16x8 ? (row & 15) + I.b * (row >> 4) : row);
            if (active && g < I.rows_per_parent) {
                const int pr = g / I.R, rr = g - pr * I.R;
                const int b = I.b, bk = I.bpow[I.k];
                const int64_t rowoff = __ldg(I.OFF + I.k * I.R + rr);
                const int cg0 = t.col0 + colbase;
                int jb = cg0 / b, c = cg0 - jb * b;
                const int nvalid = min(t.ncols - colbase, cw);
                if constexpr (OUT == TMA_OUT_F32) {
                    // FP32 output of a level k >= 1 (the all-but-one result): the columns
                    // of a row are b^k apart inside a child's block
                    float* dst = (float*)I.out + (((int64_t)t.child_base + jb) * I.P_out + pr) * I.bm + rowoff;
#pragma unroll
                    for (int e = 0; e < AW; ++e) {
                        if (e >= nvalid) break;
                        dst[(int64_t)bk * c] = acc[e];
                        if (++c == b) { c = 0; dst += I.P_out * I.bm; }
                    }
                } else if constexpr (OUT == TMA_OUT_C || OUT == TMA_OUT_C64) {
                    float* dst = (float*)I.out + (((int64_t)t.child_base + jb) * I.P_out + pr) * I.bm + rowoff;
                    // the FP32 output is C (k = 0): a row's columns are contiguous within a
                    // child's block, and b (16 or a multiple of 32) keeps groups of 4 inside blocks
                    if (((uintptr_t)I.out & 31) == 0) {
                        // 32-byte stores (a whole sector per lane): c and the row start are
                        // multiples of 8 floats, and b (a multiple of 16) keeps groups of 8
                        // inside blocks
#pragma unroll
                        for (int e = 0; e < AW; e += 8) {
                            if (e >= nvalid) break;
                            asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                                         :: "l"(dst + c), "f"((float)acc[e]), "f"((float)acc[e + 1]), "f"((float)acc[e + 2]),
                                            "f"((float)acc[e + 3]), "f"((float)acc[e + 4]), "f"((float)acc[e + 5]),
                                            "f"((float)acc[e + 6]), "f"((float)acc[e + 7])
                                         : "memory");
                            c += 8;
                            if (c == b) { c = 0; dst += I.P_out * I.bm; }
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < AW; e += 4) {
                            if (e >= nvalid) break;
                            *(float4*)(dst + c) = make_float4((float)acc[e], (float)acc[e + 1], (float)acc[e + 2],
                                                              (float)acc[e + 3]);
                            c += 4;
                            if (c == b) { c = 0; dst += I.P_out * I.bm; }
                        }
                    }
                } else {
                    // BF16 pieces of the next level's operand: [node][block][piece][b^m].
                    // Columns go in pairs (b is a multiple of 16 and a quarter starts on
                    // a multiple of 8, so a pair never straddles two children): one
                    // paired conversion per piece, one running pointer per row.
                    const int64_t bm = I.bm;
                    const int64_t child_step = (int64_t)I.P_out * NP * bm;
                    __nv_bfloat16* dst = (__nv_bfloat16*)I.out + (((int64_t)t.child_base + jb) * I.P_out + pr) * NP * bm +
                                         rowoff + (int64_t)bk * c;
                    // lanes 2i and 2i+1 hold adjacent rows (contiguous: k >= 1 and b^k >= 16):
                    // after one exchange the even lane stores column e of both rows, the odd
                    // lane column e+1, each as one 4-byte store
                    const bool odd = lane & 1;
                    const uint32_t sel = odd ? 0x3276u : 0x5410u;
                    const int64_t soff = odd ? (int64_t)bk - 1 : 0;
#pragma unroll
                    for (int e = 0; e < AW; e += 2) {
                        if (e >= nvalid) break;
                        float2 x = make_float2(acc[e], acc[e + 1]);
#pragma unroll
                        for (int pc = 0; pc < NP; ++pc) {
                            const __nv_bfloat162 h = __float22bfloat162_rn(x);
                            const uint32_t hv = *(const uint32_t*)&h;
                            const uint32_t pv = __shfl_xor_sync(0xffffffffu, hv, 1);
                            *(uint32_t*)(dst + pc * bm + soff) = __byte_perm(hv, pv, sel);
                            const float2 f = __bfloat1622float2(h);
                            x.x -= f.x;
                            x.y -= f.y;
                        }
                        c += 2;
                        if (c == b) {
                            c = 0;
                            dst += child_step - (int64_t)bk * (b - 2);
                        } else {
                            dst += 2 * (int64_t)bk;
                        }
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMAW) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_base), "r"(TCOLS));
    }
}

// FP32 BCSS -> NP BF16 pieces per block, [block][piece][b^m].
template <int NP>
__global__ void split_bcss_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int64_t nblocks, int64_t bm)
{
    const int64_t total = nblocks * bm;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t blk = i / bm, e = i - blk * bm;
        float x = in[i];
        __nv_bfloat16* o = out + blk * NP * bm + e;
#pragma unroll
        for (int pc = 0; pc < NP; ++pc) {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            o[pc * bm] = h;
            x -= __bfloat162float(h);
        }
    }
}

// The same with 8 entries per thread: two 16-byte loads, one 16-byte store per piece.
template <int NP>
__global__ void split_bcss_vec8_kernel(const float4* __restrict__ in, uint4* __restrict__ out, int64_t nblocks, int64_t bm8)
{
    const int64_t total = nblocks * bm8;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t blk = i / bm8, e = i - blk * bm8;
        const float4 x0 = in[2 * i], x1 = in[2 * i + 1];
        float v[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (int pc = 0; pc < NP; ++pc) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const __nv_bfloat16 b0 = __float2bfloat16_rn(v[2 * h]), b1 = __float2bfloat16_rn(v[2 * h + 1]);
                w[h] = pack_bf16x2(b0, b1);
                v[2 * h] -= __bfloat162float(b0);
                v[2 * h + 1] -= __bfloat162float(b1);
            }
            out[(blk * NP + pc) * bm8 + e] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

int launch_split_bcss(const float* in, void* out, int64_t nblocks, int64_t bm, int npiece, cudaStream_t s)
{
    if (npiece != 2 && npiece != 3) return (int)cudaErrorInvalidValue;
    if (bm % 8 == 0 && ((uintptr_t)in & 15) == 0 && ((uintptr_t)out & 15) == 0) {
        const int64_t total = nblocks * (bm / 8);
        int64_t g = (total + 255) / 256;
        if (g > 152 * 32) g = 152 * 32;
        if (npiece == 3) split_bcss_vec8_kernel<3><<<(int)g, 256, 0, s>>>((const float4*)in, (uint4*)out, nblocks, bm / 8);
        else split_bcss_vec8_kernel<2><<<(int)g, 256, 0, s>>>((const float4*)in, (uint4*)out, nblocks, bm / 8);
        return (int)cudaGetLastError();
    }
    const int64_t total = nblocks * bm;
    int64_t g = (total + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    if (npiece == 3) split_bcss_kernel<3><<<(int)g, 256, 0, s>>>(in, (__nv_bfloat16*)out, nblocks, bm);
    else split_bcss_kernel<2><<<(int)g, 256, 0, s>>>(in, (__nv_bfloat16*)out, nblocks, bm);
    return (int)cudaGetLastError();
}

template <int NP, int OUT, bool B, int EW>
static int launch_tma_variant(const TmaInst& inst0, const TmaInst* d_insts, const Tile* d_tiles, int ntiles, int grid,
                              int* d_status, int narrow, cudaStream_t s)
{
    constexpr int threads = (EW + 2) * 32;
    constexpr int bytes = EW == 16 ? SmemT<NP>::BYTES : SmemT<NP>::BYTES_P;
    static std::mutex mu;
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return (int)cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 0 && dev < 64 && !attr_set[dev]) {
            const cudaError_t e = cudaFuncSetAttribute(level_tma_kernel<NP, OUT, B, EW>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess) return (int)e;
            attr_set[dev] = true;
        }
    }
    level_tma_kernel<NP, OUT, B, EW><<<grid, threads, bytes, s>>>(inst0, d_insts, d_tiles, ntiles, d_status, narrow);
    return (int)cudaGetLastError();
}

// Launches of tiles <= 64 columns run the two-CTAs-per-SM form (twice the grid).
template <int NP, int OUT>
static int launch_tma_b(bool sw32, const TmaInst& inst0, const TmaInst* d_insts, const Tile* d_tiles, int ntiles,
                        int grid, int* d_status, int narrow, cudaStream_t s)
{
    if (narrow) {
        const int g2 = ntiles < 2 * grid ? ntiles : 2 * grid;
        return sw32 ? launch_tma_variant<NP, OUT, true, 8>(inst0, d_insts, d_tiles, ntiles, g2, d_status, 1, s)
                    : launch_tma_variant<NP, OUT, false, 8>(inst0, d_insts, d_tiles, ntiles, g2, d_status, 1, s);
    }
    return sw32 ? launch_tma_variant<NP, OUT, true, 16>(inst0, d_insts, d_tiles, ntiles, grid, d_status, 0, s)
               : launch_tma_variant<NP, OUT, false, 16>(inst0, d_insts, d_tiles, ntiles, grid, d_status, 0, s);
}

int launch_level_tma(int npiece, const TmaInst& inst0, const TmaInst* d_insts, const Tile* d_tiles, int ntiles,
                     int num_sms, int* d_status, int out_kind, bool sw32, int max_cols, cudaStream_t s)
{
    const int narrow = max_cols <= 64 ? 1 : 0;
    if (ntiles <= 0) return 0;
    if (npiece != 2 && npiece != 3) return (int)cudaErrorInvalidValue;
    if (out_kind < TMA_OUT_PIECES || out_kind > TMA_OUT_C64) return (int)cudaErrorInvalidValue;
    if (out_kind == TMA_OUT_C64 && max_cols > 128) return (int)cudaErrorInvalidValue;   // 32 FP64 columns per thread
    const int grid = ntiles < num_sms ? ntiles : num_sms;
    if (npiece == 2) {
        switch (out_kind) {
        case TMA_OUT_PIECES: return launch_tma_b<2, TMA_OUT_PIECES>(sw32, inst0, d_insts, d_tiles, ntiles, grid, d_status, narrow, s);
        case TMA_OUT_C: return launch_tma_b<2, TMA_OUT_C>(sw32, inst0, d_insts, d_tiles, ntiles, grid, d_status, narrow, s);
        case TMA_OUT_C64: return launch_tma_b<2, TMA_OUT_C64>(sw32, inst0, d_insts, d_tiles, ntiles, grid, d_status, narrow, s);
        default: return launch_tma_b<2, TMA_OUT_F32>(sw32, inst0, d_insts, d_tiles, ntiles, grid, d_status, narrow, s);
        }
    }
    switch (out_kind) {
    case TMA_OUT_PIECES: return launch_tma_b<3, TMA_OUT_PIECES>(sw32, inst0, d_insts, d_tiles, ntiles, grid, d_status, narrow, s);
    case TMA_OUT_C: return launch_tma_b<3, TMA_OUT_C>(sw32, inst0, d_insts, d_tiles, ntiles, grid, d_status, narrow, s);
    case TMA_OUT_C64: return launch_tma_b<3, TMA_OUT_C64>(sw32, inst0, d_insts, d_tiles, ntiles, grid, d_status, narrow, s);
    default: return launch_tma_b<3, TMA_OUT_F32>(sw32, inst0, d_insts, d_tiles, ntiles, grid, d_status, narrow, s);
    }
}

}  // namespace sttsm
