// kernels_pair.cu — the last two levels of the algorithm-by-blocks in one
// kernel for short contractions, with the temporary T^(1) kept in shared
// memory (Fig. 5, levels m-2 and m-1, with Thm. 1's partial symmetry).
//
// For a fixed parent node J of level m-2 (the sorted trailing block indices
// jb_2 <= ... <= jb_{m-1}) and fixed local trailing indices s = (j_2 ..
// j_{m-1}), the two levels are the m = 2 problem on the slice
// S_s[i0, i1] = T^(2)[J][.][i0, i1, s]:
//     U[i0, j1] = sum_{i1} S_s[i0, i1] chi_{j1, i1}          (level m-2, T^(1))
//     C[j0, j1] = sum_{i0} chi_{j0, i0} U[i0, j1],  jb_0 <= jb_1 <= jb_2   (level m-1)
// A unit of work is (J, a group of G_s consecutive s).  Its level m-2 rows
// (i0 over all nbar blocks, s in the group: nbar b G_s <= 128 rows) are
// gathered from the stored T^(2) blocks through G and the in-block offsets
// exactly as the one-level kernel gathers them; U (all children jb_1 <= jb_2
// of J at once) goes to shared memory instead of HBM; then every C block
// (jb_0 <= jb_1 <= J) of the group is contracted from U and written.  The X
// block chi[0 .. (jb_2 + 1) b, 0 .. nbar b] serves both products.
//
// Arithmetic: FP32 fused multiply-adds (two lanes per instruction), each
// output a sequential sum over the contraction index in the order the
// one-level FP32 kernel uses, so C is bit-identical to the two launches it
// replaces.  Shapes: nbar b <= 64 and pbar b <= 64.
#include <cuda_bf16.h>
#include <cstring>
#include <mutex>
#include "common.cuh"
#include "launch.h"
#include "plan.h"

namespace sttsm {

namespace {

constexpr int P_THREADS = 256;
constexpr int P_K = 64;            // contraction length bound (nbar b)
constexpr int P_N = 64;            // column bound (pbar b)
constexpr int P_ROWS = PAIR_ROWS;  // level m-2 rows per unit (nbar b G_s, with Kc G_s <= 128)
constexpr int P_U = PAIR_U_MAX;    // U entries per unit (plan.h checks every fused shape against it)

struct PairSmem {
    float A[P_K][P_ROWS];          // level m-2 operand, [k][row], row = s_local * nbar b + i0
    float X[P_K][P_N + 4];         // X[i][j] = chi_{j, i} (zero outside X)
    float U[P_U];                  // U[i0][jb1][j1 * G_s + s_local], each jb1 segment padded to 4 entries
    int32_t wsum[P_N + 1];         // level m-1 work list: first 4 x 4 block of each child jb1
};
constexpr size_t P_SMEM = sizeof(PairSmem);

template <typename Desc>
__device__ __forceinline__ const LevelInst& pair_level_of(const Desc* d, int i);
template <>
__device__ __forceinline__ const LevelInst& pair_level_of<LevelInst>(const LevelInst* d, int i) { return d[i]; }
template <>
__device__ __forceinline__ const LevelInst& pair_level_of<TcInst>(const TcInst* d, int i) { return d[i].L; }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp4(uint32_t dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_commit_wait()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void fma2(uint64_t& d, uint64_t a2, uint64_t x2)
{
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a2), "l"(x2));
}
__device__ __forceinline__ uint64_t dup2(float a)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ void split2(uint64_t v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// acc[r][c] += sum_k Aop[k][r0 + r] * Bop[k][c0 + c] for a 4 x 4 block, k < K
// (Aop rows of stride lda, Bop rows of stride ldb floats); each (r, c) is a
// sequential sum over k.
__device__ __forceinline__ void micro4x4(uint64_t acc[4][2], const float* Aop, int lda, const float* Bop, int ldb,
                                         int r0, int c0, int K)
{
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const float4 a = *(const float4*)(Aop + k * lda + r0);
        const ulonglong2 x = *(const ulonglong2*)(Bop + k * ldb + c0);
        const uint64_t a2[4] = {dup2(a.x), dup2(a.y), dup2(a.z), dup2(a.w)};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            fma2(acc[r][0], a2[r], x.x);
            fma2(acc[r][1], a2[r], x.y);
        }
    }
}

}  // namespace

// Issues the gather of a unit's level m-2 rows into S.A (cp.async; the caller
// waits): row r = sl * Kt + i0g, two threads per row taking alternate
// contraction blocks; rows past the unit and the contraction's padding to a
// multiple of 4 are zero.
__device__ __forceinline__ void pair_gather(PairSmem& S, const LevelInst& I, const Tile& t, int tid)
{
    const int b = I.b, nbar = I.nbar, R = I.R;
    const int Kt = nbar * b, Kc = (Kt + 3) & ~3;
    const int Gs = t.ncols, s0 = t.row0, S_total = R / b;
    const int rowsA = Kt * Gs;
    const int row = tid & (P_ROWS - 1), half = tid >> 7;
    const int sl = row / Kt, i0g = row - sl * Kt;
    const int s = s0 + sl;
    if (row < rowsA && s < S_total) {
        const int pr = i0g / b, rr = i0g - pr * b + b * s;
        const float* pbase = (const float*)I.parent + (int64_t)t.parent * I.P_parent * I.bm;
        const int32_t* Grow = I.G + (int64_t)pr * nbar;
        for (int ib = half; ib < nbar; ib += 2) {
            const int32_t gq = __ldg(Grow + ib);
            const int q = gq & 7;
            const int stride = I.bpow[q];
            const float* src = pbase + (int64_t)(gq >> 3) * I.bm + __ldg(I.OFF + q * R + rr);
            for (int a = 0; a < b; ++a) cp4(smem_addr(&S.A[ib * b + a][row]), src + (int64_t)a * stride);
        }
        if (half == 0)
            for (int k = Kt; k < Kc; ++k) S.A[k][row] = 0.f;
    } else {
        for (int k = half; k < Kc; k += 2) S.A[k][row] = 0.f;
    }
}

// Tile fields of a unit: parent = J (rank among level m-2 parents), row0 =
// first s of the group, ncols = G_s, col0 = children of J (jb_2 + 1, or pbar
// when m = 2), pad0 = colex-rank term of J among the C nodes (sum_t C(J_t + t
// + 2, t + 3)), inst = descriptor index.  The descriptor describes level m-2
// (k = 1; out = C).  256 threads, two CTAs per SM: two threads per gathered
// row (alternate contraction blocks), and the 4 x 4 output blocks of each
// product spread over all of them (the level m-1 blocks of every child jb_1
// of J in one list).  A CTA takes a contiguous range of units (consecutive
// units mostly share their instance's X block) and gathers the next unit's
// rows while it computes the current unit's level m-1 products.
template <typename Desc>
__global__ void __launch_bounds__(P_THREADS, 2)
level_pair_f32_kernel(const Desc* __restrict__ insts, LevelInst inst0, const Tile* __restrict__ tiles, int ntiles)
{
    extern __shared__ __align__(16) unsigned char p_raw[];
    PairSmem& S = *(PairSmem*)p_raw;
    const int tid = threadIdx.x;
    int x_inst = -1;
    // this CTA's units: a contiguous range
    const int per = ntiles / gridDim.x, extra = ntiles % gridDim.x;
    const int u_begin = blockIdx.x * per + min((int)blockIdx.x, extra);
    const int u_end = u_begin + per + ((int)blockIdx.x < extra ? 1 : 0);
    if (u_begin < u_end) {
        const Tile t0 = tiles[u_begin];
        pair_gather(S, insts ? pair_level_of(insts, t0.inst) : inst0, t0, tid);
    }
    for (int ti = u_begin; ti < u_end; ++ti) {
        const Tile t = tiles[ti];
        const LevelInst& I = insts ? pair_level_of(insts, t.inst) : inst0;
        const int b = I.b, nbar = I.nbar, R = I.R;
        const int Kt = nbar * b;                    // contraction length of both levels
        const int Kc = (Kt + 3) & ~3;
        const int Gs = t.ncols, s0 = t.row0;       // G_s (Kc G_s <= 128) and the first s of the group
        const int S_total = R / b;                  // b^(m-2) trailing index tuples
        const int rowsA = Kt * Gs;
        const int NA = t.col0 * b;                  // columns of level m-2 (all children of J)
        const int NAp = (NA + 3) & ~3;
        const int RB = b * Gs;                      // rows (j1, s) of one child jb_1 at level m-1
        const int RBp = (RB + 3) & ~3;              // its segment of U (16-byte aligned)
        const int ldU = t.col0 * RBp;               // U row stride (per i0)
        const int rbB = RBp >> 2;                   // 4-row blocks of one child at level m-1
        // ---- X block (when the instance changes): X[i][j] = chi_{j,i} for i < Kc,
        // j < pbar b rounded up to 4 (zero outside X)
        if (t.inst != x_inst) {
            const float* X = (const float*)I.X;
            const int pcols = (((I.p + b - 1) / b) * b + 3) & ~3;
            for (int e = tid; e < Kc * pcols; e += P_THREADS) {
                const int i = e / pcols, j = e - i * pcols;
                S.X[i][j] = (i < I.n && j < I.p) ? X[j + (int64_t)i * I.p] : 0.f;
            }
            x_inst = t.inst;
        }
        // ---- level m-1 work list: child jb_1 owns 4 x 4 blocks [wsum[jb_1], wsum[jb_1 + 1])
        if (tid == 0) {
            int acc = 0;
            for (int j = 0; j < t.col0; ++j) {
                S.wsum[j] = acc;
                acc += rbB * (((j + 1) * b + 3) >> 2);
            }
            S.wsum[t.col0] = acc;
        }
        cp_commit_wait();
        __syncthreads();
        // ---- level m-2: U = A^T X over rows r (4 at a time) and columns j1 (4 at a time)
        {
            const int rb = (rowsA + 3) >> 2, cb = NAp >> 2;
            for (int w = tid; w < rb * cb; w += P_THREADS) {
                const int r0 = (w % rb) * 4, c0 = (w / rb) * 4;
                uint64_t acc[4][2] = {};
                micro4x4(acc, &S.A[0][0], P_ROWS, &S.X[0][0], P_N + 4, r0, c0, Kc);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int row = r0 + r;
                    if (row >= rowsA) break;
                    const int sl = row / Kt, i0g = row - sl * Kt;
                    float v[4];
                    split2(acc[r][0], v[0], v[1]);
                    split2(acc[r][1], v[2], v[3]);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int j1g = c0 + c;
                        if (j1g >= NA) break;
                        const int jb1 = j1g / b;
                        S.U[i0g * ldU + jb1 * RBp + (j1g - jb1 * b) * Gs + sl] = v[c];
                    }
                }
            }
            // zero rows of U past the contraction (the second product reads Kc rows)
            for (int e = tid; e < (Kc - Kt) * ldU; e += P_THREADS) S.U[Kt * ldU + e] = 0.f;
        }
        __syncthreads();
        // ---- the next unit's rows, gathered while this unit's level m-1 products run
        if (ti + 1 < u_end) {
            const Tile tn = tiles[ti + 1];
            pair_gather(S, insts ? pair_level_of(insts, tn.inst) : inst0, tn, tid);
        }
        // ---- level m-1: C[j0, (j1, s)] = sum_{i0} chi_{j0,i0} U[i0, (j1, s)] for every child jb_1
        {
            const int64_t bm = I.bm;
            float* C = (float*)I.out;
            const int total = S.wsum[t.col0];
            int jb1 = 0;
            for (int w = tid; w < total; w += P_THREADS) {
                while (S.wsum[jb1 + 1] <= w) ++jb1;         // w grows, so jb_1 only moves forward
                const int local = w - S.wsum[jb1];
                const int r0 = (local % rbB) * 4, c0 = (local / rbB) * 4;
                const int NB = (jb1 + 1) * b;               // columns j0 < (jb_1 + 1) b
                uint64_t acc[4][2] = {};
                micro4x4(acc, S.U + jb1 * RBp, ldU, &S.X[0][0], P_N + 4, r0, c0, Kc);
                const int64_t cnode_base = (int64_t)t.pad0 + (int64_t)jb1 * (jb1 + 1) / 2;   // + jb_0
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int row = r0 + r;                 // row = j1 * G_s + s_local
                    if (row >= RB) break;
                    const int j1 = row / Gs, sl = row - j1 * Gs;
                    if (s0 + sl >= S_total) continue;
                    float v[4];
                    split2(acc[r][0], v[0], v[1]);
                    split2(acc[r][1], v[2], v[3]);
                    const int64_t inblk = (int64_t)b * j1 + (int64_t)b * b * (s0 + sl);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int j0g = c0 + c;
                        if (j0g >= NB) break;
                        const int jb0 = j0g / b, j0 = j0g - jb0 * b;
                        C[(cnode_base + jb0) * bm + j0 + inblk] = v[c];
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <typename Desc>
static int launch_pair(const Desc* d_insts, const LevelInst& inst0, const Tile* d_tiles, int ntiles, int num_sms,
                       cudaStream_t s)
{
    if (ntiles <= 0) return 0;
    static std::mutex mu;
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return (int)cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 0 && dev < 64 && !attr_set[dev]) {
            const cudaError_t e = cudaFuncSetAttribute(level_pair_f32_kernel<Desc>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P_SMEM);
            if (e != cudaSuccess) return (int)e;
            attr_set[dev] = true;
        }
    }
    const int grid = ntiles < num_sms * 2 ? ntiles : num_sms * 2;
    level_pair_f32_kernel<Desc><<<grid, P_THREADS, P_SMEM, s>>>(d_insts, inst0, d_tiles, ntiles);
    return (int)cudaGetLastError();
}

int launch_level_pair_f32(const LevelInst& inst0, const LevelInst* d_insts, const Tile* d_tiles, int ntiles,
                          int num_sms, cudaStream_t s)
{
    return launch_pair<LevelInst>(d_insts, inst0, d_tiles, ntiles, num_sms, s);
}

int launch_level_pair_f32_tc(const TcInst* d_insts, const Tile* d_tiles, int ntiles, int num_sms, cudaStream_t s)
{
    LevelInst none;
    memset(&none, 0, sizeof(none));
    return launch_pair<TcInst>(d_insts, none, d_tiles, ntiles, num_sms, s);
}

}  // namespace sttsm
