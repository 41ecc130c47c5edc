// kernels_tc.cu — split-precision level kernel of the algorithm-by-blocks on
// the sm_103a tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// One level of Fig. 5 with Thm. 1 (see common.cuh for the index maps): for a
// parent node and a set of unique output blocks, every child block j of the
// parent is
//     T_out[rows, j*b + c] = sum_{kk = ibar*b + a} P[rows, kk] * chi_{j*b + c, kk},
// a GEMM whose A operand P gathers rows of stored parent blocks (the
// contracted mode sits at a different local position q in each stored block,
// the permutation the paper performs explicitly before dgemm, App. A) and
// whose B operand is X itself, shared by all children of the parent.
//
// Precision: every FP32 operand is split into NP BF16 pieces
// (x = x_0 + x_1 + x_2 + rounding); the products x_s * y_t with s + t <= NP-1
// are accumulated in FP32 in tensor memory (6 products for NP = 3, 3 for NP = 2).
//
// Accumulation: the tensor core's FP32 accumulation into a large running
// sum loses low-order bits on every MMA, so the two kinds of products go to
// separate tensor-memory accumulators:
//   D0 (columns 256-511): x_0 * y_0 only, restarted every GS stages (64
//       contraction indices); the epilogue warps add each partial into an
//       FP32 register running sum (round-to-nearest);
//   D1 (columns 0-255): every cross product (s + t >= 1), accumulated over
//       the whole contraction; its values are ~2^-8 of D0's, so its rounding
//       is ~2^-8 smaller.
// The tile result is (sum of D0 partials) + D1.
//
// CTA = 17 warps, one CTA per SM, persistent over the tile list:
//   warps 0-15  workers.  Warp w serves TMEM lanes / tile rows 32 (w % 4) ..
//               +31 and chunk c = w / 4: per stage each thread gathers the 8
//               contraction entries 8c .. 8c+7 of its row with plain loads,
//               splits them into BF16 pieces and writes one 16-byte chunk per
//               piece in the SW64 K-major layout; thread 0 also issues the
//               TMA load of the X pieces.  As epilogue the warp owns the 64
//               columns 64c .. 64c+63: after producing each group it folds
//               the previous group's D0 partial into FP32 registers; at the
//               end of a tile it adds D1 and scatters the row to HBM.
//   warp 16     TMEM allocation and the single MMA-issuing thread.
// Stages: A = NP x 128 x 32 BF16, B = NP x 256 x 32 BF16, mbarrier pipeline.
// Every wait is bounded (2 s of globaltimer); on expiry the CTA records
// status 1, stops, drains, frees TMEM and returns.
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

constexpr int NUM_THREADS = 544;
constexpr int WORK_WARPS = 16;
constexpr int MMA_WARP = 16;
constexpr int GS = 2;   // stages per D0 flush group (64 contraction indices)
template <int NP>
struct Smem {
    static constexpr int A_PLANE = TC_BM * TC_KC * 2;            // 8 KB
    static constexpr int B_PLANE = TC_BN * TC_KC * 2;            // 16 KB
    static constexpr int STAGE = NP * (A_PLANE + B_PLANE);
    static constexpr int STAGES = NP == 3 ? 3 : 4;
    static constexpr int BYTES = STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/;
};

}  // namespace

// Row state of one worker thread for one tile: where its gathered A-operand
// row comes from (see common.cuh for the index maps).
struct GatherRow {
    const float* pbase;      // parent node base
    const int32_t* Grow;     // G row of the thread's output prefix block
    const int32_t* OFFrow;   // OFF + rr: off_q(rr) at OFFrow[q * R]
    bool valid;
};

// The 8 contraction entries kk0 .. kk0+7 of a row.  Within one stored block
// the entries of a row are b^q apart; with q = 0 they are contiguous and are
// read with two 16-byte loads when aligned.
__device__ __forceinline__ void gather8(const GatherRow& R, const LevelInst& I, int kk0, float* v)
{
    const int b = I.b;
    int ib = kk0 / b, a = kk0 - ib * b;
    if (!R.valid) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.f;
        return;
    }
    if (a + 8 <= b && ib < I.nbar) {
        const int32_t gq = __ldg(R.Grow + ib);
        const int q = gq & 7;
        const int bq = I.bpow[q];
        const float* src = R.pbase + (int64_t)(gq >> 3) * I.bm + __ldg(R.OFFrow + q * I.R) + (int64_t)a * bq;
        if (q == 0 && ((uintptr_t)src & 15) == 0) {
            const float4 x0 = __ldg((const float4*)src), x1 = __ldg((const float4*)src + 1);
            v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
            v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = __ldg(src + (int64_t)e * bq);
        }
        return;
    }
    // the 8 entries cross block boundaries (b < 8 or unaligned start)
    const float* src = R.pbase;
    int stride = 0;
    bool live = false;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        if (e == 0 || a == 0) {
            live = ib < I.nbar;
            if (live) {
                const int32_t gq = __ldg(R.Grow + ib);
                const int q = gq & 7;
                stride = I.bpow[q];
                src = R.pbase + (int64_t)(gq >> 3) * I.bm + __ldg(R.OFFrow + q * I.R) + (int64_t)a * stride;
            }
        }
        v[e] = live ? __ldg(src) : 0.f;
        src += stride;
        if (++a == b) { a = 0; ++ib; }
    }
}

__device__ __forceinline__ GatherRow gather_row(const Tile& t, const LevelInst& I, int row)
{
    GatherRow R;
    const int g = t.row0 + row;
    R.valid = g < I.rows_per_parent;
    const int pr = R.valid ? g / I.R : 0;
    const int rr = R.valid ? g - pr * I.R : 0;
    R.pbase = (const float*)I.parent + (int64_t)t.parent * I.P_parent * I.bm;
    R.Grow = I.G + (int64_t)pr * I.nbar;
    R.OFFrow = I.OFF + rr;
    return R;
}

// Scatter n (<= N) values of one output row into the children's blocks:
// column c0 + e goes to child (c0 + e) / b, entry (rr, (c0 + e) % b).
template <int N, typename V>
__device__ __forceinline__ void store_row(const Tile& t, const LevelInst& I, int row, int colbase, const V* vals)
{
    const int g = t.row0 + row;
    if (g >= I.rows_per_parent) return;
    const int pr = g / I.R, rr = g - pr * I.R;
    const int b = I.b, bk = I.bpow[I.k];
    const int64_t rowoff = __ldg(I.OFF + I.k * I.R + rr);
    const int cg0 = t.col0 + colbase;
    int jb = cg0 / b, c = cg0 - jb * b;
    float* dst = (float*)I.out + (((int64_t)t.child_base + jb) * I.P_out + pr) * I.bm + rowoff;
    const int nvalid = t.ncols - colbase;
    const int64_t node_stride = I.P_out * I.bm;
#pragma unroll
    for (int e = 0; e < N; ++e) {
        if (e < nvalid) dst[(int64_t)bk * c] = (float)vals[e];
        if (++c == b) { c = 0; dst += node_stride; }
    }
}

// R64: the workers' register sums are FP64 over 32 columns each (the C-block
// reduction of the R64 precisions), so tiles are at most 128 columns wide.
template <int NP, bool R64>
__global__ void __launch_bounds__(NUM_THREADS, 1)
level_tc_kernel(const __grid_constant__ TcInst inst0, const TcInst* __restrict__ insts,
                const Tile* __restrict__ tiles, int ntiles, int* status)
{
    using S = Smem<NP>;
    constexpr int STAGES = S::STAGES;
    static_assert(STAGES > GS, "producers must be able to run a whole group ahead of the flush");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + STAGES * S::STAGE);
    // bars: full[STAGES], empty[STAGES], d0_full, d0_empty, d1_empty, drain
    uint32_t* tmem_holder = (uint32_t*)(bars + 2 * STAGES + 4);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
    const uint32_t d0_full = bar0 + 8u * (2 * STAGES);
    const uint32_t d0_empty = bar0 + 8u * (2 * STAGES + 1);
    const uint32_t d1_empty = bar0 + 8u * (2 * STAGES + 2);
    const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 3);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(full_bar(s), WORK_WARPS * 32 + 1); mbar_init(empty_bar(s), 1); }
        mbar_init(d0_full, 1);
        mbar_init(d0_empty, WORK_WARPS);
        mbar_init(d1_empty, WORK_WARPS);
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(smem_u32(tmem_holder)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    const uint32_t tmem_d1 = tmem_base;
    const uint32_t tmem_d0 = tmem_base + (uint32_t)TC_BN;

    if (warp < WORK_WARPS) {
        // ------------------------------------------------------------ workers
        const int quad = warp & 3, cq = warp >> 2;
        const int row = quad * 32 + lane;                 // tile row and TMEM lane
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        constexpr int AW = R64 ? 32 : 64;                 // accumulator columns per thread
        using AccT = typename std::conditional<R64, double, float>::type;
        const int colbase = cq * AW;                      // epilogue columns
        const bool tma_thread = threadIdx.x == 0;
        int stage = 0;
        uint32_t phase = 0;
        uint32_t group_phase = 0;
        int last_stage_issued = -1;
        uint32_t last_phase_issued = 0;
        bool ok = true;
        AccT acc[AW];
        float vn[8];
        bool prefetched = false;

        // fold the D0 partial of one group into acc (all 16 warps, warp-uniform)
        auto flush = [&](bool active) -> bool {
            if (!mbar_wait(d0_full, group_phase, abort_flag, status)) return false;
            group_phase ^= 1u;
            tc_fence_after();
            if (active) {
#pragma unroll
                for (int c = 0; c < AW / 8; ++c) {
                    float v[8];
                    tmem_ld_32x32b_x8(tmem_d0 + lane_off + colbase + c * 8, v);
#pragma unroll
                    for (int i = 0; i < 8; ++i) acc[c * 8 + i] += (AccT)v[i];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(d0_empty);
            return true;
        };

        for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
            const Tile t = tiles[ti];
            const TcInst& TI = insts ? insts[t.inst] : inst0;
            const LevelInst& I = TI.L;
            const GatherRow GR = gather_row(t, I, row);
            const bool valid = GR.valid;
            const int nk = (I.Ktot + TC_KC - 1) / TC_KC;
            const bool active = colbase < t.ncols;        // warp-uniform
#pragma unroll
            for (int i = 0; i < AW; ++i) acc[i] = 0;
            if (!prefetched) gather8(GR, I, cq * 8, vn);  // stage 0 of the tile
            prefetched = false;
            for (int ks = 0; ks < nk; ++ks) {
                if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, status)) { ok = false; break; }
                uint8_t* sA = smem + stage * S::STAGE;
                uint8_t* sB = sA + NP * S::A_PLANE;
                const int k0 = ks * TC_KC;
                if (tma_thread) {
                    mbar_arrive_expect_tx(full_bar(stage), (uint32_t)(NP * S::B_PLANE));
                    tma_load_3d(smem_u32(sB), &TI.tmX, k0, t.col0, 0, full_bar(stage));
                    last_stage_issued = stage;
                    last_phase_issued = phase;
                }
                // split into BF16 pieces; piece pc goes to plane pc, row `row`,
                // 16-byte chunk cq (SW64 K-major: chunk at (cq ^ ((row >> 1) & 3)) * 16)
                const uint32_t addr0 = smem_u32(sA) + row * 64 + ((cq ^ ((row >> 1) & 3)) << 4);
#pragma unroll
                for (int pc = 0; pc < NP; ++pc) {
                    uint32_t w[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const __nv_bfloat16 b0 = __float2bfloat16_rn(vn[2 * h]), b1 = __float2bfloat16_rn(vn[2 * h + 1]);
                        w[h] = pack_bf16x2(b0, b1);
                        vn[2 * h] -= __bfloat162float(b0);
                        vn[2 * h + 1] -= __bfloat162float(b1);
                    }
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                                 :: "r"(addr0 + pc * S::A_PLANE), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]) : "memory");
                }
                fence_proxy_async();
                mbar_arrive(full_bar(stage));
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                // issue the next stage's gather; it stays in flight over the flush and the next wait
                if (ks + 1 < nk) {
                    gather8(GR, I, (ks + 1) * TC_KC + cq * 8, vn);
                } else if (ti + (int)gridDim.x < ntiles) {
                    const Tile tn = tiles[ti + gridDim.x];
                    const LevelInst& In = (insts ? insts[tn.inst] : inst0).L;
                    gather8(gather_row(tn, In, row), In, cq * 8, vn);
                    prefetched = true;
                }
                // a group is fully produced: fold the previous group's D0 partial
                if (((ks % GS) == GS - 1 || ks == nk - 1) && ks >= GS) {
                    if (!flush(active)) { ok = false; break; }
                }
            }
            if (!ok) break;
            // the last group of the tile
            if (!flush(active)) { ok = false; break; }
            // every MMA of the tile has completed (last d0_full commit): add D1
            if (active) {
#pragma unroll
                for (int c = 0; c < AW / 8; ++c) {
                    float v[8];
                    tmem_ld_32x32b_x8(tmem_d1 + lane_off + colbase + c * 8, v);
#pragma unroll
                    for (int i = 0; i < 8; ++i) acc[c * 8 + i] += (AccT)v[i];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(d1_empty);
            // scatter the row's 64 columns into the children's blocks
            if (active && valid) store_row<AW>(t, I, row, colbase, acc);
        }
        // make sure no TMA write is still in flight before the CTA exits
        if (tma_thread && !ok && last_stage_issued >= 0) {
            uint64_t t0 = globaltimer();
            while (!mbar_try_wait(full_bar(last_stage_issued), last_phase_issued))
                if (globaltimer() - t0 > WAIT_LIMIT_NS) break;
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t group_phase = 0;   // d0_empty parity counter
            uint32_t tile_phase = 0;    // d1_empty parity counter
            bool ok = true;
            bool issued = false;
            for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
                const Tile t = tiles[ti];
                const TcInst& TI = insts ? insts[t.inst] : inst0;
                const int nk = (TI.L.Ktot + TC_KC - 1) / TC_KC;
                const int nmma = (t.ncols + 15) & ~15;
                const uint32_t idesc = idesc_bf16(nmma);
                // the workers have read D1 of the previous tile
                if (!mbar_wait(d1_empty, tile_phase ^ 1u, abort_flag, status)) { ok = false; break; }
                tile_phase ^= 1u;
                tc_fence_after();
                for (int ks = 0; ks < nk; ++ks) {
                    if (!mbar_wait(full_bar(stage), phase, abort_flag, status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sA = smem_u32(smem + stage * S::STAGE);
                    const uint32_t sB = sA + NP * S::A_PLANE;
                    // cross products (s + u >= 1) into D1
#pragma unroll
                    for (int kh = 0; kh < TC_KC / 16; ++kh) {
#pragma unroll
                        for (int s = 0; s < NP; ++s) {
#pragma unroll
                            for (int u = 0; u < NP; ++u) {
                                if (s + u > NP - 1 || s + u == 0) continue;
                                const uint64_t ad = smem_desc_sw64(sA + s * S::A_PLANE + kh * 32);
                                const uint64_t bd = smem_desc_sw64(sB + u * S::B_PLANE + kh * 32);
                                const bool first = ks == 0 && kh == 0 && s == 0 && u == 1;
                                tc_mma(tmem_d1, ad, bd, idesc, first ? 0u : 1u);
                                issued = true;
                            }
                        }
                    }
                    // hi x hi into D0, restarted at each group
                    const bool group_start = (ks % GS) == 0;
                    if (group_start) {
                        if (!mbar_wait(d0_empty, group_phase ^ 1u, abort_flag, status)) { ok = false; break; }
                        group_phase ^= 1u;
                        tc_fence_after();
                    }
#pragma unroll
                    for (int kh = 0; kh < TC_KC / 16; ++kh) {
                        const uint64_t ad = smem_desc_sw64(sA + kh * 32);
                        const uint64_t bd = smem_desc_sw64(sB + kh * 32);
                        tc_mma(tmem_d0, ad, bd, idesc, (group_start && kh == 0) ? 0u : 1u);
                    }
                    tc_commit(empty_bar(stage));
                    if ((ks % GS) == GS - 1 || ks == nk - 1) tc_commit(d0_full);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok && issued) {
                // drain: wait for every MMA issued so far before TMEM is freed
                tc_commit(drain_bar);
                uint64_t t0 = globaltimer();
                while (!mbar_try_wait(drain_bar, 0))
                    if (globaltimer() - t0 > WAIT_LIMIT_NS) break;
            }
        }
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem_base));
    }
}

// ---------------------------------------------------------------------------
// Small-tile variant for launches whose contraction is short (n̄ b <= 64, at
// most two stages: one D0 group, so no register running sum is needed) —
// e.g. batches of small instances, where per-tile latency, not the tensor
// core, sets the pace.  Tiles are 128 x 64; TMEM holds two tile slots (D1,
// D0 of 64 columns each) so the MMA runs one tile ahead of the epilogue;
// 10 warps and ~110 KB of shared memory let two CTAs share an SM.
//   warps 0-7  workers: rows 32 (w % 4) .. +31; per stage each thread stores
//              the 16 contraction entries 16 (w / 4) .. +15 of its row (two
//              SW64 chunks) from a ring of three gathered stages held in
//              registers, then gathers the stage three ahead into the freed
//              slot; the epilogue of tile t-1 runs after the production of
//              tile t: columns 32 (w / 4) .. +31 of D0 + D1.
//   warp 8     TMEM allocation and the MMA-issuing thread.
//   warp 9     the X-box TMA thread, issuing each stage as soon as it frees.
constexpr int SM_THREADS = 320;
constexpr int SM_BN = 64;

template <int NP>
struct SmemSmall {
    static constexpr int A_PLANE = TC_BM * TC_KC * 2;            // 8 KB
    static constexpr int B_PLANE = SM_BN * TC_KC * 2;            // 4 KB
    static constexpr int STAGE = NP * (A_PLANE + B_PLANE);
    static constexpr int STAGES = 3;
    static constexpr int BYTES = STAGES * STAGE + 1024 + 256;
};

// Work-item cursor of the small kernel: (tile, stage) in this CTA's share.
struct ItemCursor {
    int ti, ks, nk;
};

template <int NP>
__global__ void __launch_bounds__(SM_THREADS, 2)
level_tc_small_kernel(const __grid_constant__ TcInst inst0, const TcInst* __restrict__ insts,
                      const Tile* __restrict__ tiles, int ntiles, int* status)
{
    using S = SmemSmall<NP>;
    constexpr int STAGES = S::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + STAGES * S::STAGE);
    // bars: full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], drain
    uint32_t* tmem_holder = (uint32_t*)(bars + 2 * STAGES + 5);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto accf_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + a); };
    auto acce_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + 2 + a); };
    const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(full_bar(s), 8 * 32 + 1); mbar_init(empty_bar(s), 1); }
        for (int a = 0; a < 2; ++a) { mbar_init(accf_bar(a), 1); mbar_init(acce_bar(a), 8); }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" :: "r"(smem_u32(tmem_holder)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    // slot a: D1 at columns 128 a .. +63, D0 at 128 a + 64 .. +63

    auto nk_of = [&](int ti) {
        const Tile t = tiles[ti];
        return ((insts ? insts[t.inst] : inst0).L.Ktot + TC_KC - 1) / TC_KC;
    };
    auto advance = [&](ItemCursor& c) {
        if (++c.ks == c.nk) {
            c.ti += gridDim.x;
            c.ks = 0;
            if (c.ti < ntiles) c.nk = nk_of(c.ti);
        }
    };

    if (warp < 8) {
        // ------------------------------------------------------------ workers
        const int quad = warp & 3, half = warp >> 2;
        const int row = quad * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
        const int colbase = half * 32;
        int stage = 0;
        uint32_t phase = 0, accf_phase = 0;
        bool ok = true;
        float ring[3][16];

        // epilogue of the tile pti (slot pit & 1): D0 + D1 -> the children's blocks
        auto finish = [&](int pti, int pit) -> bool {
            const int slot = pit & 1;
            if (!mbar_wait(accf_bar(slot), (accf_phase >> slot) & 1u, abort_flag, status)) return false;
            accf_phase ^= 1u << slot;
            tc_fence_after();
            const Tile t = tiles[pti];
            const LevelInst& I = (insts ? insts[t.inst] : inst0).L;
            // 8 columns at a time: TMEM loads, sum, stores (keeps few registers live)
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                if (colbase + c * 8 < t.ncols) {      // warp-uniform
                    float d0[8], d1[8];
                    tmem_ld_32x32b_x8(tmem_base + lane_off + slot * 128 + 64 + colbase + c * 8, d0);
                    tmem_ld_32x32b_x8(tmem_base + lane_off + slot * 128 + colbase + c * 8, d1);
#pragma unroll
                    for (int i = 0; i < 8; ++i) d0[i] += d1[i];
                    store_row<8>(t, I, row, colbase + c * 8, d0);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce_bar(slot));
            return true;
        };
        // gather the item of cursor g into ring slot r
        auto gather_item = [&](const ItemCursor& g, float* dst) {
            const Tile t = tiles[g.ti];
            const LevelInst& I = (insts ? insts[t.inst] : inst0).L;
            const GatherRow GR = gather_row(t, I, row);
            gather8(GR, I, g.ks * TC_KC + half * 16, dst);
            gather8(GR, I, g.ks * TC_KC + half * 16 + 8, dst + 8);
        };

        ItemCursor cc{(int)blockIdx.x, 0, 0}, gc{(int)blockIdx.x, 0, 0};
        if (cc.ti < ntiles) cc.nk = gc.nk = nk_of(cc.ti);
#pragma unroll
        for (int r = 0; r < 3; ++r)
            if (gc.ti < ntiles) { gather_item(gc, ring[r]); advance(gc); }
        int prev_ti = -1, it = 0;
        while (cc.ti < ntiles && ok) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                if (cc.ti >= ntiles || !ok) break;
                if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, status)) { ok = false; break; }
                const uint32_t sA = smem_u32(smem + stage * S::STAGE);
#pragma unroll
                for (int hc = 0; hc < 2; ++hc) {
                    float* v = ring[r] + hc * 8;
                    const int cq = half * 2 + hc;
                    const uint32_t addr0 = sA + row * 64 + ((cq ^ ((row >> 1) & 3)) << 4);
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
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                                     :: "r"(addr0 + pc * S::A_PLANE), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]) : "memory");
                    }
                }
                fence_proxy_async();
                mbar_arrive(full_bar(stage));
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                // refill this ring slot with the item three ahead
                if (gc.ti < ntiles) { gather_item(gc, ring[r]); advance(gc); }
                const int cur_ti = cc.ti;
                const bool tile_done = cc.ks + 1 == cc.nk;
                advance(cc);
                if (tile_done) {
                    // the previous tile's epilogue overlaps this tile's MMAs
                    if (prev_ti >= 0 && !finish(prev_ti, it - 1)) { ok = false; break; }
                    prev_ti = cur_ti;
                    ++it;
                }
            }
        }
        if (ok && prev_ti >= 0) ok = finish(prev_ti, it - 1);
    } else if (warp == 9) {
        // ------------------------------------------------------------ X-box producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_stage = -1;
            uint32_t last_phase = 0;
            bool ok = true;
            ItemCursor c{(int)blockIdx.x, 0, 0};
            if (c.ti < ntiles) c.nk = nk_of(c.ti);
            while (c.ti < ntiles) {
                if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, status)) { ok = false; break; }
                const Tile t = tiles[c.ti];
                const TcInst& TI = insts ? insts[t.inst] : inst0;
                const uint32_t sB = smem_u32(smem + stage * S::STAGE) + NP * S::A_PLANE;
                mbar_arrive_expect_tx(full_bar(stage), (uint32_t)(NP * S::B_PLANE));
                tma_load_3d(sB, &TI.tmX, c.ks * TC_KC, t.col0, 0, full_bar(stage));
                last_stage = stage;
                last_phase = phase;
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                advance(c);
            }
            if (!ok && last_stage >= 0) {
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(full_bar(last_stage), last_phase))
                    if (globaltimer() - t0 > WAIT_LIMIT_NS) break;
            }
        }
        __syncwarp();
    } else if (warp == 8) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, acce_phase = 0;
            bool ok = true, issued = false;
            int it = 0;
            for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x, ++it) {
                const Tile t = tiles[ti];
                const TcInst& TI = insts ? insts[t.inst] : inst0;
                const int nk = (TI.L.Ktot + TC_KC - 1) / TC_KC;
                const uint32_t idesc = idesc_bf16((t.ncols + 15) & ~15);
                const int slot = it & 1;
                if (!mbar_wait(acce_bar(slot), ((acce_phase >> slot) & 1u) ^ 1u, abort_flag, status)) { ok = false; break; }
                acce_phase ^= 1u << slot;
                tc_fence_after();
                const uint32_t d1 = tmem_base + slot * 128, d0 = d1 + 64;
                for (int ks = 0; ks < nk; ++ks) {
                    if (!mbar_wait(full_bar(stage), phase, abort_flag, status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sA = smem_u32(smem + stage * S::STAGE);
                    const uint32_t sB = sA + NP * S::A_PLANE;
#pragma unroll
                    for (int kh = 0; kh < TC_KC / 16; ++kh) {
#pragma unroll
                        for (int s = 0; s < NP; ++s) {
#pragma unroll
                            for (int u = 0; u < NP; ++u) {
                                if (s + u > NP - 1) continue;
                                const uint64_t ad = smem_desc_sw64(sA + s * S::A_PLANE + kh * 32);
                                const uint64_t bd = smem_desc_sw64(sB + u * S::B_PLANE + kh * 32);
                                const bool first = ks == 0 && kh == 0 && (s + u == 0 || (s == 0 && u == 1));
                                tc_mma(s + u == 0 ? d0 : d1, ad, bd, idesc, first ? 0u : 1u);
                                issued = true;
                            }
                        }
                    }
                    tc_commit(empty_bar(stage));
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                tc_commit(accf_bar(slot));
            }
            if (!ok && issued) {
                tc_commit(drain_bar);
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(drain_bar, 0))
                    if (globaltimer() - t0 > WAIT_LIMIT_NS) break;
            }
        }
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 8) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" :: "r"(tmem_base));
    }
}

int launch_level_tc_small(int npiece, const TcInst& inst0, const TcInst* d_insts, const Tile* d_tiles, int ntiles,
                          int num_sms, int* d_status, cudaStream_t s)
{
    if (ntiles <= 0) return 0;
    const int grid = ntiles < 2 * num_sms ? ntiles : 2 * num_sms;
    static std::mutex mu;
    static bool attr_set[2][64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (npiece != 2 && npiece != 3) return (int)cudaErrorInvalidValue;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 0 && dev < 64 && !attr_set[npiece - 2][dev]) {
            cudaError_t e = npiece == 3
                ? cudaFuncSetAttribute(level_tc_small_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SmemSmall<3>::BYTES)
                : cudaFuncSetAttribute(level_tc_small_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SmemSmall<2>::BYTES);
            if (e != cudaSuccess) return (int)e;
            attr_set[npiece - 2][dev] = true;
        }
    }
    if (npiece == 3)
        level_tc_small_kernel<3><<<grid, SM_THREADS, SmemSmall<3>::BYTES, s>>>(inst0, d_insts, d_tiles, ntiles, d_status);
    else
        level_tc_small_kernel<2><<<grid, SM_THREADS, SmemSmall<2>::BYTES, s>>>(inst0, d_insts, d_tiles, ntiles, d_status);
    return (int)cudaGetLastError();
}

template <int NP, bool R64>
static int launch_tc_variant(const TcInst& inst0, const TcInst* d_insts, const Tile* d_tiles, int ntiles, int grid,
                             int* d_status, cudaStream_t s)
{
    // the shared-memory opt-in is set once per device (never inside a stream capture after the first call)
    static std::mutex mu;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 0 && dev < 64 && !attr_set[dev]) {
            const cudaError_t e = cudaFuncSetAttribute(level_tc_kernel<NP, R64>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<NP>::BYTES);
            if (e != cudaSuccess) return (int)e;
            attr_set[dev] = true;
        }
    }
    level_tc_kernel<NP, R64><<<grid, NUM_THREADS, Smem<NP>::BYTES, s>>>(inst0, d_insts, d_tiles, ntiles, d_status);
    return (int)cudaGetLastError();
}

int launch_level_tc(int npiece, const TcInst& inst0, const TcInst* d_insts, const Tile* d_tiles, int ntiles,
                    int num_sms, int* d_status, cudaStream_t s)
{
    if (ntiles <= 0) return 0;
    const int grid = ntiles < num_sms ? ntiles : num_sms;
    if (npiece == 3) return launch_tc_variant<3, false>(inst0, d_insts, d_tiles, ntiles, grid, d_status, s);
    if (npiece == 2) return launch_tc_variant<2, false>(inst0, d_insts, d_tiles, ntiles, grid, d_status, s);
    return (int)cudaErrorInvalidValue;
}

int launch_level_tc_r64(int npiece, const TcInst& inst0, const TcInst* d_insts, const Tile* d_tiles, int ntiles,
                        int num_sms, int* d_status, int max_cols, cudaStream_t s)
{
    if (ntiles <= 0) return 0;
    if (max_cols > 128) return (int)cudaErrorInvalidValue;   // 32 FP64 columns per worker
    const int grid = ntiles < num_sms ? ntiles : num_sms;
    if (npiece == 3) return launch_tc_variant<3, true>(inst0, d_insts, d_tiles, ntiles, grid, d_status, s);
    if (npiece == 2) return launch_tc_variant<2, true>(inst0, d_insts, d_tiles, ntiles, grid, d_status, s);
    return (int)cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ bounded-wait probe

// One thread waits on an mbarrier that no thread ever arrives on, with the
// same bounded-wait loop the level kernels use but a caller-given limit; on
// timeout it raises the status word exactly as a level kernel would, and the
// CTA leaves.  It exercises the failure path without faulting the GPU.
__global__ void wait_probe_kernel(int* status, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = ptx::smem_u32(&bar);
    ptx::mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!ptx::mbar_wait_for(b, 0, limit_ns)) atomicExch(status, 1);
}

int launch_wait_probe(int* d_status, unsigned long long limit_ns, cudaStream_t s)
{
    wait_probe_kernel<<<1, 32, 0, s>>>(d_status, limit_ns);
    return (int)cudaGetLastError();
}

}  // namespace sttsm
