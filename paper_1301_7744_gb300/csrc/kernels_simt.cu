// kernels_simt.cu — CUDA-core kernels: BCSS pack/unpack (Sec. 3.3, 5.3),
// the FP32 -> BF16-piece split of X, and the plain FP64 level kernel of the
// algorithm-by-blocks (Fig. 5 with Thm. 1).
#include <cuda_bf16.h>
#include "common.cuh"
#include "launch.h"

namespace sttsm {

// ------------------------------------------------------------------ pack / unpack

// One CTA per stored block (grid-stride): the block's sorted tuple is
// unranked once, then the b^m entries are copied with entry e = in-block
// dimensional offset; consecutive e read consecutive dense addresses.
template <typename T>
__global__ void bcss_pack_kernel(const T* __restrict__ dense, T* __restrict__ bcss, int m, int64_t n, int b,
                                 int64_t nblocks, int64_t bm)
{
    __shared__ int32_t tup[STTSM_MAX_M];
    for (int64_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) colex_unrank(blk, m, tup);
        __syncthreads();
        T* dst = bcss + blk * bm;
        for (int64_t e = threadIdx.x; e < bm; e += blockDim.x) {
            int64_t r = e, off = 0, stride = 1;
            bool inside = true;
            for (int a = 0; a < m; ++a) {
                int64_t i = (int64_t)tup[a] * b + r % b;
                r /= b;
                inside = inside && (i < n);
                off += i * stride;
                stride *= n;
            }
            dst[e] = inside ? dense[off] : T(0);
        }
    }
}

// One thread per dense entry: sort the indices, read the canonical entry.
template <typename T>
__global__ void bcss_unpack_kernel(const T* __restrict__ bcss, T* __restrict__ dense, int m, int64_t n, int b,
                                   int64_t total, int64_t bm)
{
    for (int64_t lin = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lin < total;
         lin += (int64_t)gridDim.x * blockDim.x) {
        int32_t s[STTSM_MAX_M];
        int64_t r = lin;
        for (int a = 0; a < m; ++a) { s[a] = (int32_t)(r % n); r /= n; }
        for (int a = 1; a < m; ++a) {  // insertion sort, m <= 8
            int32_t v = s[a];
            int c = a - 1;
            while (c >= 0 && s[c] > v) { s[c + 1] = s[c]; --c; }
            s[c + 1] = v;
        }
        int32_t blk[STTSM_MAX_M];
        int64_t loc = 0, w = 1;
        for (int a = 0; a < m; ++a) {
            blk[a] = s[a] / b;
            loc += (int64_t)(s[a] % b) * w;
            w *= b;
        }
        dense[lin] = bcss[colex_rank(blk, m) * bm + loc];
    }
}

int launch_bcss_pack(const void* dense, void* bcss, int m, int64_t n, int b, int dtype, cudaStream_t s)
{
    int64_t nbar = (n + b - 1) / b;
    int64_t nblocks = binom_small(nbar + m - 1, m);
    int64_t bm = 1;
    for (int a = 0; a < m; ++a) bm *= b;
    int threads = bm >= 256 ? 256 : (bm >= 64 ? 64 : 32);
    int64_t g = nblocks < 152 * 64 ? nblocks : 152 * 64;
    if (dtype == 0) bcss_pack_kernel<double><<<(int)g, threads, 0, s>>>((const double*)dense, (double*)bcss, m, n, b, nblocks, bm);
    else bcss_pack_kernel<float><<<(int)g, threads, 0, s>>>((const float*)dense, (float*)bcss, m, n, b, nblocks, bm);
    return (int)cudaGetLastError();
}

int launch_bcss_unpack(const void* bcss, void* dense, int m, int64_t n, int b, int dtype, cudaStream_t s)
{
    int64_t total = 1, bm = 1;
    for (int a = 0; a < m; ++a) { total *= n; bm *= b; }
    int64_t g = (total + 255) / 256;
    if (g > 152 * 64) g = 152 * 64;
    if (dtype == 0) bcss_unpack_kernel<double><<<(int)g, 256, 0, s>>>((const double*)bcss, (double*)dense, m, n, b, total, bm);
    else bcss_unpack_kernel<float><<<(int)g, 256, 0, s>>>((const float*)bcss, (float*)dense, m, n, b, total, bm);
    return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ X split

// X (p x n, column-major FP32) -> npiece BF16 planes [piece][rows][Kp], row j
// holding chi_{j, 0..n-1} (K-major operand rows), zero beyond p and n.
// Piece t is the BF16 rounding of what pieces 0..t-1 left over.
__global__ void split_x_kernel(const float* __restrict__ X, __nv_bfloat16* __restrict__ out, int p, int n,
                               int rows, int Kp, int npiece)
{
    int64_t total = (int64_t)rows * Kp;
    int64_t plane = total;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int j = (int)(t / Kp), i = (int)(t % Kp);
        float v = (j < p && i < n) ? X[j + (int64_t)i * p] : 0.f;
        for (int pc = 0; pc < npiece; ++pc) {
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            out[pc * plane + t] = h;
            v = v - __bfloat162float(h);
        }
    }
}

int launch_split_x(const float* X, void* out, int p, int n, int rows, int Kp, int npiece, cudaStream_t s)
{
    int64_t total = (int64_t)rows * Kp;
    int64_t g = (total + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    split_x_kernel<<<(int)g, 256, 0, s>>>(X, (__nv_bfloat16*)out, p, n, rows, Kp, npiece);
    return (int)cudaGetLastError();
}

__global__ void split_x_batch_kernel(const SplitDesc* __restrict__ d, int count, int npiece)
{
    // this CTA's instance: the last descriptor with first_block <= blockIdx.x
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (d[mid].first_block <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const SplitDesc D = d[lo];
    const int64_t total = (int64_t)D.rows * D.Kp;
    const int64_t t = ((int64_t)blockIdx.x - D.first_block) * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int j = (int)(t / D.Kp), i = (int)(t % D.Kp);
    float v = (j < D.p && i < D.n) ? D.X[j + (int64_t)i * D.p] : 0.f;
    __nv_bfloat16* out = (__nv_bfloat16*)D.out;
    for (int pc = 0; pc < npiece; ++pc) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        out[pc * total + t] = h;
        v = v - __bfloat162float(h);
    }
}

int launch_split_x_batch(const SplitDesc* d_desc, int count, int blocks, int npiece, cudaStream_t s)
{
    if (count <= 0 || blocks <= 0) return 0;
    split_x_batch_kernel<<<blocks, 256, 0, s>>>(d_desc, count, npiece);
    return (int)cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 level kernel

// Tile of 64 output rows x 64 output columns, 256 threads, each thread 4x4
// results, contraction index kk in chunks of 16 staged through shared memory.
// The gathered operand (rows of stored parent blocks, Thm. 1) and X are read
// with the index maps documented in common.cuh.
constexpr int F64_BM = 64, F64_BN = 64, F64_BK = 16;

__global__ void __launch_bounds__(256)
level_fp64_kernel(const LevelInst* __restrict__ insts, LevelInst inst0, const Tile* __restrict__ tiles, int ntiles)
{
    __shared__ double As[F64_BK][F64_BM + 1];
    __shared__ double Xs[F64_BK][F64_BN + 1];
    const int tid = threadIdx.x;
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile t = tiles[ti];
        const LevelInst& I = insts ? insts[t.inst] : inst0;
        const double* parent = (const double*)I.parent + (int64_t)t.parent * I.P_parent * I.bm;
        const double* X = (const double*)I.X;
        // loader role: row lr of the tile, contraction offsets lk0..lk0+3
        const int lr = tid & 63, lk0 = (tid >> 6) * 4;
        const int64_t lg = (int64_t)t.row0 + lr;
        const bool lvalid = lg < I.rows_per_parent;
        const int lpr = lvalid ? (int)(lg / I.R) : 0;
        const int lrr = lvalid ? (int)(lg % I.R) : 0;
        // X loader role: column xc, same contraction offsets
        const int xc = tid & 63;
        const int xj = t.col0 + xc;
        const bool xvalid = (xc < t.ncols) && (xj < I.p);
        double acc[4][4] = {};
        const int ty = tid >> 4, tx = tid & 15;
        for (int k0 = 0; k0 < I.Ktot; k0 += F64_BK) {
            __syncthreads();
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int kk = k0 + lk0 + e;
                double v = 0.0;
                if (lvalid && kk < I.Ktot) {
                    const int ib = kk / I.b, a = kk - ib * I.b;
                    const int32_t g = I.G[(int64_t)lpr * I.nbar + ib];
                    const int q = g & 7;
                    const int64_t rank = g >> 3;
                    const int bq = I.bpow[q];
                    const int64_t off = I.OFF[q * I.R + lrr] + (int64_t)a * bq;
                    v = parent[rank * I.bm + off];
                }
                As[lk0 + e][lr] = v;
                double xv = 0.0;
                if (xvalid && kk < I.n) xv = X[xj + (int64_t)kk * I.p];
                Xs[lk0 + e][xc] = xv;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < F64_BK; ++kk) {
                double av[4], xv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) xv[j] = Xs[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], xv[j], acc[i][j]);
            }
        }
        // epilogue: scatter the 4x4 results into the children's blocks
        double* out = (double*)I.out;
        const int bk = I.bpow[I.k];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t g = (int64_t)t.row0 + ty * 4 + i;
            if (g >= I.rows_per_parent) continue;
            const int pr = (int)(g / I.R), rr = (int)(g % I.R);
            const int64_t rowoff = I.OFF[I.k * I.R + rr];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = tx * 4 + j;
                if (col >= t.ncols) continue;
                const int cg = t.col0 + col;
                const int jb = cg / I.b, c = cg - jb * I.b;
                const int64_t node = (int64_t)t.child_base + jb;
                out[(node * I.P_out + pr) * I.bm + rowoff + (int64_t)bk * c] = acc[i][j];
            }
        }
    }
}

int launch_level_fp64(const LevelInst& inst0, const LevelInst* d_insts, const Tile* d_tiles, int ntiles,
                      int num_sms, cudaStream_t s)
{
    if (ntiles <= 0) return 0;
    int grid = ntiles < num_sms * 8 ? ntiles : num_sms * 8;
    level_fp64_kernel<<<grid, 256, 0, s>>>(d_insts, inst0, d_tiles, ntiles);
    return (int)cudaGetLastError();
}

}  // namespace sttsm
