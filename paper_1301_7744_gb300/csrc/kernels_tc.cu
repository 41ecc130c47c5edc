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
// CTA = 9 warps, one CTA per SM, persistent over the tile list:
//   warps 0-3  epilogue: tcgen05.ld of the 128 x N FP32 tile, scatter to HBM;
//   warps 4-7  producers: thread t gathers row t of the A tile (32 contraction
//              indices per stage) with plain loads, splits it into BF16
//              pieces and writes them in the SW64 K-major layout;
//              thread 128 also issues the TMA load of the X pieces;
//   warp 8     TMEM allocation and the single MMA-issuing thread.
// Stages: A = NP x 128 x 32 BF16, B = NP x 256 x 32 BF16, mbarrier pipeline;
// two TMEM accumulators (2 x 256 columns) overlap epilogue and MMA.
// Every wait is bounded (2 s of globaltimer); on expiry the CTA records
// status 1, stops, drains, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda.h>
#include "common.cuh"
#include "launch.h"

namespace sttsm {

namespace {

constexpr int NUM_THREADS = 288;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and raises the CTA abort flag) on timeout or
// when another role already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag) return false;
            uint64_t now = globaltimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > WAIT_LIMIT_NS) {
                *abort_flag = 1;
                atomicExch(status, 1);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum) : "memory");
}

// 32 lanes x 32 consecutive FP32 columns; thread i receives lane (base + i).
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (16-byte units), fixed version bits 46-48 = 0b001,
// swizzle mode in bits 61-63 (4 = 64-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;   // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n (multiple of 16, <= 256).
__device__ __forceinline__ uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <int NP>
struct Smem {
    static constexpr int A_PLANE = TC_BM * TC_KC * 2;            // 8 KB
    static constexpr int B_PLANE = TC_BN * TC_KC * 2;            // 16 KB
    static constexpr int STAGE = NP * (A_PLANE + B_PLANE);
    static constexpr int STAGES = NP == 3 ? 3 : 4;
    static constexpr int BYTES = STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/;
};

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

}  // namespace

template <int NP>
__global__ void __launch_bounds__(NUM_THREADS, 1)
level_tc_kernel(const __grid_constant__ TcInst inst0, const TcInst* __restrict__ insts,
                const Tile* __restrict__ tiles, int ntiles, int* status)
{
    using S = Smem<NP>;
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
        for (int s = 0; s < STAGES; ++s) { mbar_init(full_bar(s), 129); mbar_init(empty_bar(s), 1); }
        for (int a = 0; a < 2; ++a) { mbar_init(accf_bar(a), 1); mbar_init(acce_bar(a), 128); }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(smem_u32(tmem_holder)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    if (warp >= 4 && warp < 8) {
        // ------------------------------------------------------------ producers
        const int pt = threadIdx.x - 128;                // row of the A tile
        const bool tma_thread = (pt == 0);
        int stage = 0;
        uint32_t phase = 0;
        int last_stage_issued = -1;
        uint32_t last_phase_issued = 0;
        bool ok = true;
        for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
            const Tile t = tiles[ti];
            const TcInst& TI = insts ? insts[t.inst] : inst0;
            const LevelInst& I = TI.L;
            const float* pbase = (const float*)I.parent + (int64_t)t.parent * I.P_parent * I.bm;
            const int64_t g = (int64_t)t.row0 + pt;
            const bool valid = g < I.rows_per_parent;
            const int pr = valid ? (int)(g / I.R) : 0;
            const int rr = valid ? (int)(g % I.R) : 0;
            const int32_t* Grow = I.G + (int64_t)pr * I.nbar;
            const int b = I.b, nbar = I.nbar;
            const int nk = (I.Ktot + TC_KC - 1) / TC_KC;
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
                // gather 32 contraction entries of this row
                float v[TC_KC];
                int ib = k0 / b, a = k0 - ib * b;
                const float* src = pbase;
                int64_t stride = 0;
                bool live = false;
                auto seg = [&]() {
                    live = valid && ib < nbar;
                    if (live) {
                        const int32_t gq = __ldg(Grow + ib);
                        const int q = gq & 7;
                        const int64_t rank = gq >> 3;
                        const int bq = I.bpow[q];
                        stride = bq;
                        src = pbase + rank * I.bm + (rr % bq) + (int64_t)bq * b * (rr / bq) + (int64_t)a * bq;
                    }
                };
                seg();
#pragma unroll
                for (int e = 0; e < TC_KC; ++e) {
                    v[e] = live ? __ldg(src) : 0.f;
                    if (live) src += stride;
                    if (++a == b) { a = 0; ++ib; seg(); }
                }
                // split into BF16 pieces and store the row (SW64 K-major: row r
                // at r*64 B, 16-byte chunk c at (c ^ ((r >> 1) & 3)) * 16)
                const uint32_t rowbase = smem_u32(sA) + pt * 64;
                const int sw = (pt >> 1) & 3;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    uint32_t w[NP][4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        float x0 = v[c * 8 + 2 * h], x1 = v[c * 8 + 2 * h + 1];
#pragma unroll
                        for (int pc = 0; pc < NP; ++pc) {
                            __nv_bfloat16 b0 = __float2bfloat16_rn(x0), b1 = __float2bfloat16_rn(x1);
                            w[pc][h] = pack_bf16x2(b0, b1);
                            x0 -= __bfloat162float(b0);
                            x1 -= __bfloat162float(b1);
                        }
                    }
#pragma unroll
                    for (int pc = 0; pc < NP; ++pc) {
                        const uint32_t addr = rowbase + pc * S::A_PLANE + ((c ^ sw) << 4);
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                                     :: "r"(addr), "r"(w[pc][0]), "r"(w[pc][1]), "r"(w[pc][2]), "r"(w[pc][3]) : "memory");
                    }
                }
                fence_proxy_async();
                mbar_arrive(full_bar(stage));
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
        }
        // make sure no TMA write is still in flight before the CTA exits
        if (tma_thread && !ok && last_stage_issued >= 0) {
            uint64_t t0 = globaltimer();
            while (!mbar_try_wait(full_bar(last_stage_issued), last_phase_issued))
                if (globaltimer() - t0 > WAIT_LIMIT_NS) break;
        }
    } else if (warp == 8) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t acc_phase = 0;   // bit a = phase of accumulator a
            int acc = 0;
            bool ok = true;
            bool issued = false;
            for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
                const Tile t = tiles[ti];
                const TcInst& TI = insts ? insts[t.inst] : inst0;
                const int nk = (TI.L.Ktot + TC_KC - 1) / TC_KC;
                const int nmma = (t.ncols + 15) & ~15;
                const uint32_t idesc = idesc_bf16(nmma);
                if (!mbar_wait(acce_bar(acc), ((acc_phase >> acc) & 1u) ^ 1u, abort_flag, status)) { ok = false; break; }
                tc_fence_after();
                const uint32_t tmem_d = tmem_base + (uint32_t)(acc * TC_BN);
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
                                const uint32_t accum = (ks > 0 || kh > 0 || s > 0 || u > 0) ? 1u : 0u;
                                tc_mma(tmem_d, ad, bd, idesc, accum);
                                issued = true;
                            }
                        }
                    }
                    tc_commit(empty_bar(stage));
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                tc_commit(accf_bar(acc));
                acc_phase ^= 1u << acc;
                acc ^= 1;
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
    } else {
        // ------------------------------------------------------------ epilogue (warps 0-3)
        const int row = warp * 32 + lane;
        uint32_t acc_phase = 0;   // bit a = phase of accumulator a
        int acc = 0;
        for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
            const Tile t = tiles[ti];
            const TcInst& TI = insts ? insts[t.inst] : inst0;
            const LevelInst& I = TI.L;
            if (!mbar_wait(accf_bar(acc), (acc_phase >> acc) & 1u, abort_flag, status)) break;
            tc_fence_after();
            const int64_t g = (int64_t)t.row0 + row;
            const bool valid = g < I.rows_per_parent;
            const int pr = valid ? (int)(g / I.R) : 0;
            const int rr = valid ? (int)(g % I.R) : 0;
            const int bk = I.bpow[I.k];
            const int b = I.b;
            float* out = (float*)I.out;
            const int64_t rowoff = (rr % bk) + (int64_t)bk * b * (rr / bk);
            const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * TC_BN);
            for (int c0 = 0; c0 < t.ncols; c0 += 32) {
                float v[32];
                tmem_ld_32x32b_x32(taddr + c0, v);
                if (valid) {
                    int cg = t.col0 + c0;
                    int jb = cg / b, c = cg - jb * b;
                    float* dst = out + (((int64_t)t.child_base + jb) * I.P_out + pr) * I.bm + rowoff;
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        if (c0 + e < t.ncols) dst[(int64_t)bk * c] = v[e];
                        if (++c == b) { c = 0; ++jb; dst += I.P_out * I.bm; }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acce_bar(acc));
            acc_phase ^= 1u << acc;
            acc ^= 1;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 8) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem_base));
    }
}

int launch_level_tc(int npiece, const TcInst& inst0, const TcInst* d_insts, const Tile* d_tiles, int ntiles,
                    int num_sms, int* d_status, cudaStream_t s)
{
    if (ntiles <= 0) return 0;
    const int grid = ntiles < num_sms ? ntiles : num_sms;
    if (npiece == 3) {
        cudaError_t e = cudaFuncSetAttribute(level_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<3>::BYTES);
        if (e != cudaSuccess) return (int)e;
        level_tc_kernel<3><<<grid, NUM_THREADS, Smem<3>::BYTES, s>>>(inst0, d_insts, d_tiles, ntiles, d_status);
    } else if (npiece == 2) {
        cudaError_t e = cudaFuncSetAttribute(level_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<2>::BYTES);
        if (e != cudaSuccess) return (int)e;
        level_tc_kernel<2><<<grid, NUM_THREADS, Smem<2>::BYTES, s>>>(inst0, d_insts, d_tiles, ntiles, d_status);
    } else {
        return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

}  // namespace sttsm
