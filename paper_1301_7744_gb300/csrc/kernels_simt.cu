// kernels_simt.cu — CUDA-core kernels: BCSS pack/unpack (Sec. 3.3, 5.3),
// the FP32 -> BF16-piece split of X, and the plain FP64 level kernel of the
// algorithm-by-blocks (Fig. 5 with Thm. 1).
#include <cuda_bf16.h>
#include <cstddef>
#include <cstring>
#include <type_traits>
#include <mutex>
#include "common.cuh"
#include "sym.cuh"
#include "launch.h"

namespace sttsm {

// ------------------------------------------------------------------ pack / unpack

// Work unit = (stored block, chunk of PACK_CHUNK in-block entries), grid-
// stride, so that even few large blocks (b = 64: 364 blocks of 262144
// entries) keep every SM busy.  The unit's block tuple is unranked once; entry
// e = in-block dimensional offset, consecutive e read consecutive dense
// addresses.  The digits of e are taken with 32-bit division when
// b^m < 2^31 (64-bit otherwise).
constexpr int64_t PACK_CHUNK = 8192;

template <typename T, typename IT>
__device__ __forceinline__ void bcss_pack_range(const T* __restrict__ dense, T* __restrict__ dst, const int32_t* tup,
                                                int m, int64_t n, int b, int lb, IT e0, IT e1)
{
#pragma unroll 4
    for (IT e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        IT r = e;
        int64_t off = 0, stride = 1;
        bool inside = true;
        for (int a = 0; a < m; ++a) {
            const IT q = lb >= 0 ? (IT)(r >> lb) : r / (IT)b;   // lb = log2 b when b is a power of two
            const int64_t i = (int64_t)tup[a] * b + (int64_t)(r - q * (IT)b);
            r = q;
            inside = inside && (i < n);
            off += i * stride;
            stride *= n;
        }
        dst[e] = inside ? dense[off] : T(0);
    }
}

// The same with V consecutive entries per thread (one 16-byte load and store):
// when b and n are multiples of V, entries e .. e + V - 1 (e a multiple of V)
// share every index but i_0 and are V consecutive dense entries, all inside
// or all outside the tensor.
template <typename T, int V, typename IT>
__device__ __forceinline__ void bcss_pack_range_vec(const T* __restrict__ dense, T* __restrict__ dst,
                                                    const int32_t* tup, int m, int64_t n, int b, int lb, IT e0, IT e1)
{
    using W = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
#pragma unroll 2
    for (IT e = e0 + (IT)threadIdx.x * V; e < e1; e += (IT)blockDim.x * V) {
        IT r = e;
        int64_t off = 0, stride = 1;
        bool inside = true;
        for (int a = 0; a < m; ++a) {
            const IT q = lb >= 0 ? (IT)(r >> lb) : r / (IT)b;
            const int64_t i = (int64_t)tup[a] * b + (int64_t)(r - q * (IT)b);
            r = q;
            inside = inside && (i < n);
            off += i * stride;
            stride *= n;
        }
        W v;
        if (inside) v = *(const W*)(dense + off);
        else memset(&v, 0, sizeof(v));
        *(W*)(dst + e) = v;
    }
}

template <typename T>
__global__ void bcss_pack_kernel(const T* __restrict__ dense, T* __restrict__ bcss, int m, int64_t n, int b,
                                 int64_t nblocks, int64_t bm, int vec)
{
    __shared__ int32_t tup[STTSM_MAX_M];
    const int64_t nchunk = (bm + PACK_CHUNK - 1) / PACK_CHUNK;
    const int lb = (b & (b - 1)) == 0 ? __ffs(b) - 1 : -1;
    for (int64_t w = blockIdx.x; w < nblocks * nchunk; w += gridDim.x) {
        const int64_t blk = w / nchunk, c0 = (w - blk * nchunk) * PACK_CHUNK;
        const int64_t c1 = c0 + PACK_CHUNK < bm ? c0 + PACK_CHUNK : bm;
        __syncthreads();
        if (threadIdx.x == 0) colex_unrank(blk, m, tup);
        __syncthreads();
        T* dst = bcss + blk * bm;
        constexpr int V = 16 / sizeof(T);
        if (vec && bm < ((int64_t)1 << 31))
            bcss_pack_range_vec<T, V, uint32_t>(dense, dst, tup, m, n, b, lb, (uint32_t)c0, (uint32_t)c1);
        else if (vec)
            bcss_pack_range_vec<T, V, int64_t>(dense, dst, tup, m, n, b, lb, c0, c1);
        else if (bm < ((int64_t)1 << 31))
            bcss_pack_range<T, uint32_t>(dense, dst, tup, m, n, b, lb, (uint32_t)c0, (uint32_t)c1);
        else
            bcss_pack_range<T, int64_t>(dense, dst, tup, m, n, b, lb, c0, c1);
    }
}

// The same work units for the common case (16-byte accesses, b^M < 2^31,
// M * nbar colex-rank terms fit in shared memory), with the order M a template
// parameter: every thread unranks the unit's block tuple itself from the
// tabulated terms C(v + t, t + 1) (a binary search per position; no barrier
// per unit), and the per-entry loops have exactly M steps.
template <typename T, int M>
__global__ void __launch_bounds__(256)
bcss_pack_vec_kernel(const T* __restrict__ dense, T* __restrict__ bcss, int64_t n, int b, int nbar, int64_t nblocks,
                     uint32_t bm)
{
    using W = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    constexpr int V = 16 / sizeof(T);
    extern __shared__ int64_t pk_ctab[];   // pk_ctab[t * nbar + v] = C(v + t, t + 1)
    for (int i = threadIdx.x; i < M * nbar; i += blockDim.x) {
        const int t = i / nbar, v = i - t * nbar;
        pk_ctab[i] = binom_small((int64_t)v + t, t + 1);
    }
    __syncthreads();
    const bool bpow2 = (b & (b - 1)) == 0;
    const int lb = bpow2 ? __ffs(b) - 1 : 0;
    int64_t npow[M];
    {
        int64_t w = 1;
#pragma unroll
        for (int a = 0; a < M; ++a) { npow[a] = w; w *= n; }
    }
    int top = 1;   // largest power of two <= nbar
    while (top * 2 <= nbar) top *= 2;
    const uint32_t nchunk = (bm + (uint32_t)PACK_CHUNK - 1) / (uint32_t)PACK_CHUNK;
    for (int64_t w = blockIdx.x; w < nblocks * nchunk; w += gridDim.x) {
        const int64_t blk = w / nchunk;
        const uint32_t c0 = (uint32_t)(w - blk * nchunk) * (uint32_t)PACK_CHUNK;
        const uint32_t c1 = c0 + (uint32_t)PACK_CHUNK < bm ? c0 + (uint32_t)PACK_CHUNK : bm;
        int32_t tup[M];
        {
            int64_t r = blk;
#pragma unroll
            for (int t = M - 1; t >= 0; --t) {
                const int64_t* ct = pk_ctab + t * nbar;
                int v = 0;
                for (int step = top; step > 0; step >>= 1)
                    if (v + step < nbar && ct[v + step] <= r) v += step;
                tup[t] = v;
                r -= ct[v];
            }
        }
        T* dst = bcss + blk * (int64_t)bm;
#pragma unroll 2
        for (uint32_t e = c0 + threadIdx.x * V; e < c1; e += blockDim.x * V) {
            uint32_t r = e;
            int64_t off = 0;
            bool inside = true;
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const uint32_t q = bpow2 ? r >> lb : r / (uint32_t)b;
                const int64_t i = (int64_t)tup[a] * b + (int64_t)(r - q * (uint32_t)b);
                r = q;
                inside = inside && (i < n);
                off += i * npow[a];
            }
            W v;
            if (inside) v = *(const W*)(dense + off);
            else memset(&v, 0, sizeof(v));
            *(W*)(dst + e) = v;
        }
    }
}

// One thread per dense entry: sort the indices (a compare-exchange network on
// registers), read the canonical entry.  The colex rank of the sorted block
// tuple sums C(v_t + t, t + 1) over its positions t; with tab the CTA first
// tabulates those terms for every position and block index in shared memory
// (m * nbar entries), otherwise each is computed.
template <typename T>
__global__ void bcss_unpack_kernel(const T* __restrict__ bcss, T* __restrict__ dense, int m, int64_t n, int b,
                                   int64_t total, int64_t bm, int nbar, int tab)
{
    extern __shared__ int64_t ctab[];   // ctab[t * nbar + v] = C(v + t, t + 1)
    if (tab) {
        for (int i = threadIdx.x; i < m * nbar; i += blockDim.x) {
            const int t = i / nbar, v = i - t * nbar;
            ctab[i] = binom_small((int64_t)v + t, t + 1);
        }
        __syncthreads();
    }
    const int64_t rest_total = m > 1 ? total / n : 1;
    const bool small = rest_total < ((int64_t)1 << 31);
    const bool small_lin = total < ((int64_t)1 << 32);
    const int lb = (b & (b - 1)) == 0 ? __ffs(b) - 1 : -1;
    for (int64_t lin = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lin < total;
         lin += (int64_t)gridDim.x * blockDim.x) {
        int32_t s[STTSM_MAX_M];
        int64_t r0;
        if (small_lin) {
            const uint32_t l = (uint32_t)lin, q = l / (uint32_t)n;
            r0 = q;
            s[0] = (int32_t)(l - q * (uint32_t)n);
        } else {
            r0 = lin / n;
            s[0] = (int32_t)(lin - r0 * n);
        }
        if (small) {
            uint32_t r = (uint32_t)r0;
            const uint32_t un = (uint32_t)n;
#pragma unroll
            for (int a = 1; a < STTSM_MAX_M; ++a) {
                if (a < m) { const uint32_t q = r / un; s[a] = (int32_t)(r - q * un); r = q; }
            }
        } else {
            int64_t r = r0;
#pragma unroll
            for (int a = 1; a < STTSM_MAX_M; ++a) {
                if (a < m) { s[a] = (int32_t)(r % n); r /= n; }
            }
        }
        // bubble network over s[0 .. m-1], fixed indices so s stays in registers
#pragma unroll
        for (int i = 0; i < STTSM_MAX_M - 1; ++i) {
#pragma unroll
            for (int j = 0; j < STTSM_MAX_M - 1 - i; ++j) {
                if (j + 1 < m - i) {
                    const int32_t lo = min(s[j], s[j + 1]), hi = max(s[j], s[j + 1]);
                    s[j] = lo;
                    s[j + 1] = hi;
                }
            }
        }
        int64_t rank = 0, loc = 0, w = 1;
#pragma unroll
        for (int a = 0; a < STTSM_MAX_M; ++a) {
            if (a < m) {
                const int32_t v = lb >= 0 ? (s[a] >> lb) : s[a] / b;
                rank += tab ? ctab[a * nbar + v] : binom_small((int64_t)v + a, a + 1);
                loc += (int64_t)(s[a] - v * b) * w;
                w *= b;
            }
        }
        dense[lin] = bcss[rank * bm + loc];
    }
}

// Unpack by tiles (m >= 2).  A work unit is one dense block B (block indices
// B_0 .. B_{m-1}, any order), a TX x TX tile of in-block offsets along dense
// mode 0 (x) and along mode a* (y; the mode >= 1 holding the smallest block),
// and a group of S consecutive slabs of the other m - 2 offsets.  Every entry
// reads from the stored block sort(B) (rank once per unit), at the offsets of
// its sorted full indices (the canonical entry; a sort of M values per entry).
// The reads go along whichever of x and y is stored mode 0 (B_0 the strict
// minimum: x; else y), so a warp reads consecutive stored entries, through a
// padded shared tile; the writes go along x, consecutive dense entries.  The
// unit first tabulates its slabs' fixed offsets (8 bits each, b <= 256) and
// their share of the dense address in shared memory.  The order M is a
// template parameter so the per-entry loops and the sorting network have
// exactly M (M (M-1) / 2) steps; in-block offsets are 32-bit (b^M < 2^31).
constexpr int UT_MAX_SLABS = 256;

template <typename T, int M>
__global__ void __launch_bounds__(256)
bcss_unpack_tiled_kernel(const T* __restrict__ bcss, T* __restrict__ dense, int64_t n, int b, int nbar, int64_t bm,
                         int TX, int ntx, int slabs, int S, uint32_t ngrp, uint32_t total_units, int vec4)
{
    extern __shared__ __align__(16) unsigned char ut_raw[];
    int64_t* ctab = (int64_t*)ut_raw;                             // ctab[t * nbar + v] = C(v + t, t + 1)
    int64_t* slab_addr = ctab + (size_t)M * nbar;                 // [S] dense-address share of the slab's offsets
    uint64_t* slab_off = (uint64_t*)(slab_addr + UT_MAX_SLABS);   // [S] offsets of modes != 0, a* (8 bits each)
    T* tile = (T*)(slab_off + UT_MAX_SLABS);                      // [S][TX][TX + 1]
    for (int i = threadIdx.x; i < M * nbar; i += blockDim.x) {
        const int t = i / nbar, v = i - t * nbar;
        ctab[i] = binom_small((int64_t)v + t, t + 1);
    }
    const int P = TX + 1;
    const bool tpow2 = (TX & (TX - 1)) == 0;
    const int ltx = tpow2 ? __ffs(TX) - 1 : 0;
    const bool bpow2 = (b & (b - 1)) == 0;
    const int lb = bpow2 ? __ffs(b) - 1 : 0;
    const uint32_t per_block = (uint32_t)(ntx * ntx) * ngrp;
    for (uint32_t u = blockIdx.x; u < total_units; u += gridDim.x) {
        const uint32_t blin = u / per_block;
        uint32_t rem = u - blin * per_block;
        const uint32_t tt = rem / ngrp;
        const int slab0 = (int)(rem - tt * ngrp) * S;
        const int tyi = (int)tt / ntx, txi = (int)tt - tyi * ntx;
        const int nslab = slabs - slab0 < S ? slabs - slab0 : S;
        int32_t B[M], sB[M];
        {
            uint32_t r = blin;
#pragma unroll
            for (int a = 0; a < M; ++a) {
                const uint32_t q = r / (uint32_t)nbar;
                B[a] = (int32_t)(r - q * (uint32_t)nbar);
                sB[a] = B[a];
                r = q;
            }
        }
        int as = 1, Bas = B[1];
#pragma unroll
        for (int a = 2; a < M; ++a)
            if (B[a] < Bas) { as = a; Bas = B[a]; }
        const bool read_x = B[0] < Bas;
#pragma unroll
        for (int i = 0; i < M - 1; ++i)
#pragma unroll
            for (int j = 0; j < M - 1 - i; ++j) {
                const int32_t lo = min(sB[j], sB[j + 1]), hi = max(sB[j], sB[j + 1]);
                sB[j] = lo;
                sB[j + 1] = hi;
            }
        int64_t nas = 1;   // n^a*
        for (int a = 0; a < as; ++a) nas *= n;
        const int x0 = txi * TX, y0 = tyi * TX;
        const int nx = b - x0 < TX ? b - x0 : TX, ny = b - y0 < TX ? b - y0 : TX;
        const int64_t bx = (int64_t)B[0] * b + x0, by = (int64_t)Bas * b + y0;
        const int xlim = n - bx < nx ? (int)(n - bx) : nx;   // x < xlim: index < n
        const int ylim = n - by < ny ? (int)(n - by) : ny;
        const int64_t base = bx + by * nas;
        __syncthreads();   // ctab filled (first unit) / the previous unit is done with the tables and the tile
        if (xlim <= 0 || ylim <= 0) continue;   // uniform in the CTA
        int64_t rank = 0;
#pragma unroll
        for (int a = 0; a < M; ++a) rank += ctab[a * nbar + sB[a]];
        const T* src = bcss + rank * bm;
        // no repeated block index: mode a goes to stored mode pi(a) = #{B_a' < B_a} for
        // every entry, so the stored offset is linear in the tile's coordinates
        uint32_t wpi[M];   // b^pi(a)
        bool tiefree = true;
#pragma unroll
        for (int a = 0; a < M; ++a) {
            int pa = 0;
#pragma unroll
            for (int a2 = 0; a2 < M; ++a2) {
                pa += B[a2] < B[a] ? 1 : 0;
                tiefree = tiefree && (a2 == a || B[a2] != B[a]);
            }
            uint32_t w = 1;
            for (int t = 0; t < pa; ++t) w *= (uint32_t)b;
            wpi[a] = w;
        }
        const bool fast = vec4 && tiefree;
        for (int sl = threadIdx.x; sl < nslab; sl += blockDim.x) {
            uint32_t sr = (uint32_t)(slab0 + sl);
            int64_t share = 0, w = 1;
            uint64_t offs = 0;
            bool ok = true;
            int c = 0;
#pragma unroll
            for (int a = 0; a < M; ++a) {
                if (a > 0 && a != as) {
                    const uint32_t q = bpow2 ? sr >> lb : sr / (uint32_t)b;
                    const int off = (int)(sr - q * (uint32_t)b);
                    sr = q;
                    const int64_t i = (int64_t)B[a] * b + off;
                    ok = ok && i < n;
                    share += i * w;
                    if (fast) offs += (uint64_t)((uint32_t)off * wpi[a]);
                    else offs |= (uint64_t)off << (8 * c);
                    ++c;
                }
                w *= n;
            }
            slab_addr[sl] = ok ? share : -1;
            slab_off[sl] = offs;   // fast: the fixed modes' share of the stored offset
        }
        __syncthreads();
        if (fast) {
            // 4 consecutive entries per access (b, n, TX multiples of 4; 16-byte aligned arrays)
            const int TX4 = TX >> 2;
            const int cnt4 = nslab * TX * TX4;
            const uint32_t corner = (uint32_t)x0 * wpi[0] + (uint32_t)y0 * wpi[as];   // the tile's origin
            if (read_x) {
                // x is stored mode 0 and dense mode 0: a straight copy along x
                const uint32_t wy = wpi[as];
                for (int e = threadIdx.x; e < cnt4; e += blockDim.x) {
                    const int sl = e / (TX * TX4), w = e - sl * TX * TX4;
                    const int y = w / TX4, x = (w - y * TX4) * 4;
                    const int64_t sa = slab_addr[sl];
                    if (x >= xlim || y >= ylim || sa < 0) continue;
                    const float4 v = *(const float4*)((const float*)src + corner + (uint32_t)slab_off[sl] + x + y * wy);
                    *(float4*)((float*)dense + base + sa + x + (int64_t)y * nas) = v;
                }
                continue;
            }
            // y is stored mode 0: 4 consecutive y in, transposed in the tile, 4 consecutive x out
            const uint32_t wx = wpi[0];
            for (int e = threadIdx.x; e < cnt4; e += blockDim.x) {
                const int sl = e / (TX * TX4), w = e - sl * TX * TX4;
                const int x = w / TX4, y = (w - x * TX4) * 4;
                if (x >= xlim || y >= ylim || slab_addr[sl] < 0) continue;
                const float4 v = *(const float4*)((const float*)src + corner + (uint32_t)slab_off[sl] + x * wx + y);
                float* tp = (float*)tile + (sl * TX + x) * P + y;
                tp[0] = v.x;
                tp[1] = v.y;
                tp[2] = v.z;
                tp[3] = v.w;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < cnt4; e += blockDim.x) {
                const int sl = e / (TX * TX4), w = e - sl * TX * TX4;
                const int y = w / TX4, x = (w - y * TX4) * 4;
                const int64_t sa = slab_addr[sl];
                if (x >= xlim || y >= ylim || sa < 0) continue;
                const float* tp = (const float*)tile + (sl * TX + x) * P + y;
                *(float4*)((float*)dense + base + sa + x + (int64_t)y * nas) = make_float4(tp[0], tp[P], tp[2 * P], tp[3 * P]);
            }
            continue;
        }
        // in-block offset of sorted full indices s_t: sum_t s_t b^t - sum_t sB_t b^(t+1),
        // below b^M < 2^31; the terms wrap modulo 2^32 (unsigned), the difference is exact
        uint32_t bmul[M];   // b^t
        {
            uint32_t w = 1;
#pragma unroll
            for (int a = 0; a < M; ++a) { bmul[a] = w; w *= (uint32_t)b; }
        }
        uint32_t sbase = 0;
#pragma unroll
        for (int a = 0; a < M; ++a) sbase += (uint32_t)sB[a] * (uint32_t)b * bmul[a];
        const int cnt = nslab * TX * TX;
        if (vec4) {
            // 4 consecutive entries along the read axis per iteration: one decode, four
            // canonical-entry sorts and four independent loads
            const int TX4 = TX >> 2;
            const int cnt4 = nslab * TX * TX4;
            const int lim_a = read_x ? xlim : ylim, lim_b = read_x ? ylim : xlim;   // limits along fa, fb
            const int va = read_x ? 0 : as;   // the mode along which the 4 entries run
            for (int e = threadIdx.x; e < cnt4; e += blockDim.x) {
                const int sl = e / (TX * TX4), w = e - sl * TX * TX4;
                const int fb = w / TX4, fa0 = (w - fb * TX4) * 4;
                if (fa0 >= lim_a || fb >= lim_b || slab_addr[sl] < 0) continue;
                const uint64_t offs = slab_off[sl];
                int32_t f0[M];
                int c = 0;
#pragma unroll
                for (int a = 0; a < M; ++a) {
                    if (a == 0) {
                        f0[a] = (int32_t)bx + (read_x ? fa0 : fb);
                    } else if (a == as) {
                        f0[a] = (int32_t)by + (read_x ? fb : fa0);
                    } else {
                        f0[a] = B[a] * b + (int)((offs >> (8 * c)) & 255);
                        ++c;
                    }
                }
                T v4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    int32_t f[M];
#pragma unroll
                    for (int a = 0; a < M; ++a) f[a] = f0[a] + (a == va ? u : 0);
#pragma unroll
                    for (int i = 0; i < M - 1; ++i)
#pragma unroll
                        for (int j = 0; j < M - 1 - i; ++j) {
                            const int32_t lo = min(f[j], f[j + 1]), hi = max(f[j], f[j + 1]);
                            f[j] = lo;
                            f[j + 1] = hi;
                        }
                    uint32_t loc = 0u - sbase;
#pragma unroll
                    for (int a = 0; a < M; ++a) loc += (uint32_t)f[a] * bmul[a];
                    v4[u] = src[loc];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int x = read_x ? fa0 + u : fb, y = read_x ? fb : fa0 + u;
                    tile[(sl * TX + x) * P + y] = v4[u];
                }
            }
        } else
#pragma unroll 4
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            int sl, w;
            if (tpow2) { sl = e >> (2 * ltx); w = e & (TX * TX - 1); }
            else { sl = e / (TX * TX); w = e - sl * TX * TX; }
            const int fa = tpow2 ? (w & (TX - 1)) : w % TX, fb = tpow2 ? (w >> ltx) : w / TX;
            const int x = read_x ? fa : fb, y = read_x ? fb : fa;
            if (x >= xlim || y >= ylim || slab_addr[sl] < 0) continue;
            const uint64_t offs = slab_off[sl];
            int32_t f[M];
            int c = 0;
#pragma unroll
            for (int a = 0; a < M; ++a) {
                if (a == 0) {
                    f[a] = (int32_t)bx + x;
                } else if (a == as) {
                    f[a] = (int32_t)by + y;
                } else {
                    f[a] = B[a] * b + (int)((offs >> (8 * c)) & 255);
                    ++c;
                }
            }
#pragma unroll
            for (int i = 0; i < M - 1; ++i)
#pragma unroll
                for (int j = 0; j < M - 1 - i; ++j) {
                    const int32_t lo = min(f[j], f[j + 1]), hi = max(f[j], f[j + 1]);
                    f[j] = lo;
                    f[j + 1] = hi;
                }
            uint32_t loc = 0u - sbase;
#pragma unroll
            for (int a = 0; a < M; ++a) loc += (uint32_t)f[a] * bmul[a];
            tile[(sl * TX + x) * P + y] = src[loc];
        }
        __syncthreads();
        if (vec4) {
            // the write side does not depend on the block: 4 consecutive x per store
            const int TX4 = TX >> 2;
            const int cnt4 = nslab * TX * TX4;
            for (int e = threadIdx.x; e < cnt4; e += blockDim.x) {
                const int sl = e / (TX * TX4), w = e - sl * TX * TX4;
                const int y = w / TX4, x = (w - y * TX4) * 4;
                const int64_t sa = slab_addr[sl];
                if (x >= xlim || y >= ylim || sa < 0) continue;
                const float* tp = (const float*)tile + (sl * TX + x) * P + y;
                *(float4*)((float*)dense + base + sa + x + (int64_t)y * nas) = make_float4(tp[0], tp[P], tp[2 * P], tp[3 * P]);
            }
            continue;
        }
#pragma unroll 4
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            int sl, w;
            if (tpow2) { sl = e >> (2 * ltx); w = e & (TX * TX - 1); }
            else { sl = e / (TX * TX); w = e - sl * TX * TX; }
            const int x = tpow2 ? (w & (TX - 1)) : w % TX, y = tpow2 ? (w >> ltx) : w / TX;
            const int64_t sa = slab_addr[sl];
            if (x >= xlim || y >= ylim || sa < 0) continue;
            dense[base + sa + x + (int64_t)y * nas] = tile[(sl * TX + x) * P + y];
        }
    }
}

template <typename T>
static int launch_unpack_tiled(const T* bcss, T* dense, int m, int64_t n, int b, int nbar, int64_t bm, int TX,
                               int ntx, int slabs, int S, uint32_t ngrp, uint32_t total_units, size_t smem,
                               cudaStream_t s)
{
    // 16-byte accesses for blocks without a repeated index: FP32, b, n and TX multiples
    // of 4, both arrays 16-byte aligned
    const int vec4 = (sizeof(T) == 4 && b % 4 == 0 && n % 4 == 0 && TX % 4 == 0 && ((uintptr_t)bcss & 15) == 0 &&
                      ((uintptr_t)dense & 15) == 0) ? 1 : 0;
    const int g = (int)(total_units < 152u * 8u ? total_units : 152u * 8u);
    switch (m) {
#define UT_CASE(MM)                                                                                             \
    case MM:                                                                                                    \
        bcss_unpack_tiled_kernel<T, MM><<<g, 256, smem, s>>>(bcss, dense, n, b, nbar, bm, TX, ntx, slabs, S,    \
                                                             ngrp, total_units, vec4);                          \
        break;
        UT_CASE(2) UT_CASE(3) UT_CASE(4) UT_CASE(5) UT_CASE(6) UT_CASE(7) UT_CASE(8)
#undef UT_CASE
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

int launch_bcss_pack(const void* dense, void* bcss, int m, int64_t n, int b, int dtype, cudaStream_t s)
{
    int64_t nbar = (n + b - 1) / b;
    int64_t nblocks = binom_small(nbar + m - 1, m);
    int64_t bm = 1;
    for (int a = 0; a < m; ++a) bm *= b;
    int threads = bm >= 256 ? 256 : (bm >= 64 ? 64 : 32);
    const int64_t work = nblocks * ((bm + PACK_CHUNK - 1) / PACK_CHUNK);
    int64_t g = work < 152 * 64 ? work : 152 * 64;
    // 16-byte accesses: V = 4 floats or 2 doubles per thread when b and n are
    // multiples of V and both arrays are 16-byte aligned (chunks are multiples of V)
    const int V = dtype == 0 ? 2 : 4;
    const int vec = (b % V == 0 && n % V == 0 && ((uintptr_t)dense & 15) == 0 && ((uintptr_t)bcss & 15) == 0) ? 1 : 0;
    const size_t ctab_bytes = (size_t)m * nbar * sizeof(int64_t);
    if (vec && m >= 1 && bm < ((int64_t)1 << 31) && ctab_bytes <= 32768) {
        const int gg = (int)g;
        const int nb = (int)nbar;
        switch (m) {
#define PK_CASE(MM)                                                                                                 \
    case MM:                                                                                                        \
        if (dtype == 0)                                                                                             \
            bcss_pack_vec_kernel<double, MM><<<gg, threads, ctab_bytes, s>>>((const double*)dense, (double*)bcss, n, b, \
                                                                          nb, nblocks, (uint32_t)bm);               \
        else                                                                                                        \
            bcss_pack_vec_kernel<float, MM><<<gg, threads, ctab_bytes, s>>>((const float*)dense, (float*)bcss, n, b, nb, \
                                                                         nblocks, (uint32_t)bm);                    \
        return (int)cudaGetLastError();
            PK_CASE(1) PK_CASE(2) PK_CASE(3) PK_CASE(4) PK_CASE(5) PK_CASE(6) PK_CASE(7) PK_CASE(8)
#undef PK_CASE
        default: break;
        }
    }
    if (dtype == 0)
        bcss_pack_kernel<double><<<(int)g, threads, 0, s>>>((const double*)dense, (double*)bcss, m, n, b, nblocks, bm, vec);
    else
        bcss_pack_kernel<float><<<(int)g, threads, 0, s>>>((const float*)dense, (float*)bcss, m, n, b, nblocks, bm, vec);
    return (int)cudaGetLastError();
}

int launch_bcss_unpack(const void* bcss, void* dense, int m, int64_t n, int b, int dtype, cudaStream_t s)
{
    int64_t total = 1, bm = 1;
    for (int a = 0; a < m; ++a) { total *= n; bm *= b; }
    const int64_t nbar = (n + b - 1) / b;
    // rank terms tabulated in shared memory when they fit in 32 KB
    const size_t tab_bytes = (size_t)m * (size_t)nbar * sizeof(int64_t);
    const int tab = tab_bytes <= 32768 ? 1 : 0;
    const size_t smem = tab ? tab_bytes : 0;
    if (m >= 2 && b <= 256 && bm < ((int64_t)1 << 31)) {
        // units: dense block x tile of TX x TX offsets (modes 0 and a*) x group of S slabs
        // TX: b below 32, else the largest power of two <= 32 dividing b (no partial tiles)
        int TX = b < 32 ? b : 32;
        while (b >= 32 && b % TX != 0) TX >>= 1;
        // b between 32 and 64 that 32 does not divide (48, ...): one tile the block's width
        // (rows of b, not 16, contiguous floats; 0.425 -> 0.49 of HBM at b = 48)
        if (b > 32 && b < 64 && b % 32 != 0 && b % 4 == 0 && dtype == 1) TX = b;
        const int ntx = (b + TX - 1) / TX;
        int64_t slabs = 1;
        for (int a = 2; a < m; ++a) slabs *= b;
        // groups of up to 8192 entries (several loads in flight per thread between
        // barriers), tile <= 36 KB
        const size_t esz = dtype == 0 ? sizeof(double) : sizeof(float);
        int S = 8192 / (TX * TX);
        const int s_bytes = (int)(36864 / ((size_t)TX * (TX + 1) * esz));
        if (S > s_bytes) S = s_bytes;
        if (S < 1) S = 1;
        if ((int64_t)S > slabs) S = (int)slabs;
        if (S > UT_MAX_SLABS) S = UT_MAX_SLABS;
        const int64_t ngrp = (slabs + S - 1) / S;
        int64_t nblk = 1;
        for (int a = 0; a < m; ++a) nblk *= nbar;
        const int64_t total_units = nblk * ntx * ntx * ngrp;
        const size_t smem2 = (size_t)m * nbar * sizeof(int64_t) + (size_t)UT_MAX_SLABS * 16 +
                             (size_t)S * TX * (TX + 1) * esz;
        if (smem2 <= 48 * 1024 && total_units < ((int64_t)1 << 31)) {
            if (dtype == 0)
                return launch_unpack_tiled<double>((const double*)bcss, (double*)dense, m, n, b, (int)nbar, bm, TX,
                                                   ntx, (int)slabs, S, (uint32_t)ngrp, (uint32_t)total_units, smem2, s);
            return launch_unpack_tiled<float>((const float*)bcss, (float*)dense, m, n, b, (int)nbar, bm, TX, ntx,
                                              (int)slabs, S, (uint32_t)ngrp, (uint32_t)total_units, smem2, s);
        }
    }
    int64_t g = (total + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (dtype == 0)
        bcss_unpack_kernel<double><<<(int)g, 256, smem, s>>>((const double*)bcss, (double*)dense, m, n, b, total, bm,
                                                              (int)nbar, tab);
    else
        bcss_unpack_kernel<float><<<(int)g, 256, smem, s>>>((const float*)bcss, (float*)dense, m, n, b, total, bm,
                                                             (int)nbar, tab);
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

// ------------------------------------------------------------------ FP32 small-contraction kernel

// Level kernel for short contractions (n̄ b <= 64) in FP32 on the CUDA cores,
// one thread per output row of a 128 x <=64 tile.  A CTA stages one tile at
// a time in shared memory with cp.async (the tile's A rows, gathered from the
// stored parent blocks through G and the in-block offsets off_q, computed
// with shifts for b in {4, 8, 16} and read from the OFF table otherwise, and
// its X block); four CTAs share an SM, so the copies of one overlap the
// arithmetic of the others.  A CTA copies an X block only when it differs
// from the one of its previous tile.
// Both operands are kept [kk][...] in shared memory: A[kk][row] (the 4-byte
// copies of 32 rows and the reads of a contraction row are conflict-free),
// X[kk][column] read by broadcast.  The column count of a tile selects a
// compile-time width (8, 16, 24, 32, 48 or 64), so the inner loop has no
// predicates, and a register blocking (1, 2 or 4 rows per thread) that
// lets one X read feed several rows; column pairs accumulate through the
// two-lane FMA.  Results of b a power of two >= 4 are stored four columns at a
// time (one 16-byte store at k = 0).  Every entry is a sequential FP32 sum of
// <= 64 products.
// Used where tensor-core tiles of <= 64 columns and <= 64 contraction indices
// are latency-bound (batches and serving of small instances).
constexpr int S32_ROWS = 128, S32_COLS = 64, S32_K = 64;

// Tiles in the in-block-symmetry mode (sym.cuh): tile row t is the parent's
// canonical row rho = row0 + t, at row g[t] = pr * R + rr of the full row map
// (-1 past the parent's canonical rows), tie[t] its runs of equal blocks,
// blk[t] its i blocks (8 bits each).
struct S32Sym {
    SymTab tab;
    int32_t g[S32_ROWS];
    uint32_t tie[S32_ROWS];
    uint32_t blk[S32_ROWS];
};
struct S32Stage {
    float A[S32_K][S32_ROWS];         // A[kk][t]: operand of output row row0 + t (canonical row g[t])
    float X[S32_K][S32_COLS];         // X[kk][c] = chi_{col0 + c, kk}, zero outside the tile / X
    S32Sym sym;
};
constexpr int S32_CTAS_PER_SM = 4;
constexpr size_t S32_SMEM = sizeof(S32Stage);

template <typename Desc>
__device__ __forceinline__ const LevelInst& level_of(const Desc* d, int i);
template <>
__device__ __forceinline__ const LevelInst& level_of<LevelInst>(const LevelInst* d, int i) { return d[i]; }
template <>
__device__ __forceinline__ const LevelInst& level_of<TcInst>(const TcInst* d, int i) { return d[i].L; }

__device__ __forceinline__ uint32_t s32_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void s32_cp4(uint32_t dst, const void* src, int bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void s32_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void s32_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ int s32_width_class(int ncols)
{
    return ncols <= 8 ? 0 : ncols <= 16 ? 1 : ncols <= 24 ? 2 : ncols <= 32 ? 3 : ncols <= 48 ? 4 : 5;
}

// Column offset of contraction row kk of a tile's X block: a warp copies
// 32 / NCX rows at once (NCX = NC rounded up to a power of two), and rows
// 64 words apart share banks, so rows of tiles <= 8 (<= 16) columns wide are
// shifted by 8 (kk mod 4) (16 (kk mod 2)) words.  The compute loop steps kk
// by 4, so the shift of row kk + u is known at compile time.
template <int NC>
__host__ __device__ constexpr int s32_xshift(int kk)
{
    return NC <= 8 ? 8 * (kk & 3) : (NC <= 16 ? 16 * (kk & 1) : 0);
}

// X block of a tile (zero-filled outside the tile and outside X).  Lane
// t copies column t mod NCX of rows t / NCX, t / NCX + 128 / NCX, ...
template <int NC>
__device__ __forceinline__ void s32_issue_x(S32Stage& S, const LevelInst& I, const Tile& t, int Kc)
{
    constexpr int NCX = NC <= 8 ? 8 : NC <= 16 ? 16 : NC <= 32 ? 32 : 64;
    constexpr int KSTEP = S32_ROWS / NCX;
    const float* X = (const float*)I.X;
    const int c = threadIdx.x & (NCX - 1);
    const int j = t.col0 + c;
    const bool colok = c < t.ncols && j < I.p;
    const int nrows = colok ? (I.n < Kc ? I.n : Kc) : 0;
    const int64_t pstep = (int64_t)KSTEP * I.p;
    int kk = threadIdx.x / NCX;
    const float* src = X + j + (int64_t)kk * I.p;
    // the shift is the same for all rows of this thread (KSTEP is a multiple of 4)
    uint32_t dst = s32_smem(&S.X[kk][c + s32_xshift<NC>(kk)]);
    for (; kk < nrows; kk += KSTEP, src += pstep, dst += KSTEP * S32_COLS * 4) s32_cp4(dst, src, 4);
    for (; kk < Kc; kk += KSTEP, dst += KSTEP * S32_COLS * 4) s32_cp4(dst, X, 0);
}

// b entries of one contraction block (source stride b^q, compile-time for
// B > 0) into consecutive contraction rows of the stage
constexpr int S32_KROW = S32_ROWS * 4;   // bytes between contraction rows of A
template <int B, int STRIDE>
__device__ __forceinline__ void s32_copy_block(uint32_t dst, const float* src)
{
#pragma unroll
    for (int a = 0; a < B; ++a) s32_cp4(dst + S32_KROW * a, src + a * STRIDE, 4);
}

template <int B>
__device__ __forceinline__ void s32_copy_q(uint32_t dst, const float* src, int q)
{
    switch (q) {
    case 1: s32_copy_block<B, B>(dst, src); break;
    case 2: s32_copy_block<B, B * B>(dst, src); break;
    case 3: s32_copy_block<B, B * B * B>(dst, src); break;
    case 4: s32_copy_block<B, B * B * B * B>(dst, src); break;
    default: {
        int stride = 1;
        for (int i = 0; i < q; ++i) stride *= B;
#pragma unroll
        for (int a = 0; a < B; ++a) s32_cp4(dst + S32_KROW * a, src + (int64_t)a * stride, 4);
    }
    }
}

// Operand row of this thread: for every contraction block ib the stored
// parent block rank(sort(prefix + ib)) and the insertion position q give the
// entries off_q(rr) + a b^q, a = 0..b-1 (Thm. 1).  B > 0: b == B (strides
// known at compile time); B == 0: any b.
template <int B>
__device__ __forceinline__ void s32_issue_a(S32Stage& S, const LevelInst& I, const Tile& t, int Kc)
{
    const int g = t.row0 + threadIdx.x;
    if (g >= I.rows_per_parent) return;
    const int R = I.R, b = B > 0 ? B : I.b, nbar = I.nbar;
    const int64_t bm = I.bm;
    const int32_t* OFF = I.OFF;
    const int pr = g / R, rr = g - pr * R;
    const float* pbase = (const float*)I.parent + (int64_t)t.parent * I.P_parent * bm;
    const int32_t* Grow = I.G + (int64_t)pr * nbar;
    // 16 contraction blocks per round (more only when b < 4); the table
    // loads of a round are issued together
    for (int ib0 = 0; ib0 < nbar; ib0 += S32_K / 4) {
        int32_t gq[S32_K / 4];
        int32_t off[S32_K / 4];
#pragma unroll
        for (int i = 0; i < S32_K / 4; ++i) gq[i] = ib0 + i < nbar ? __ldg(Grow + ib0 + i) : 0;
        if (B > 0) {
            // off_q(rr) = rr mod b^q + b^(q+1) (rr div b^q), b = 2^LB
            constexpr int LB = B == 4 ? 2 : (B == 8 ? 3 : 4);
#pragma unroll
            for (int i = 0; i < S32_K / 4; ++i) {
                const int lq = (gq[i] & 7) * LB;
                off[i] = (rr & ((1 << lq) - 1)) + ((rr >> lq) << (lq + LB));
            }
        } else {
#pragma unroll
            for (int i = 0; i < S32_K / 4; ++i) off[i] = ib0 + i < nbar ? __ldg(OFF + (gq[i] & 7) * R + rr) : 0;
        }
#pragma unroll
        for (int i = 0; i < S32_K / 4; ++i) {
            if (ib0 + i >= nbar) break;
            const int q = gq[i] & 7;
            const float* src = pbase + (int64_t)(gq[i] >> 3) * bm + off[i];
            const uint32_t d0 = s32_smem(&S.A[(ib0 + i) * b][threadIdx.x]);
            if (B > 0) {
                if (q == 0) s32_copy_block<(B > 0 ? B : 1), 1>(d0, src);
                else s32_copy_q<(B > 0 ? B : 1)>(d0, src, q);
            } else {
                const int stride = I.bpow[q];
#pragma unroll 4
                for (int a = 0; a < b; ++a) s32_cp4(d0 + S32_KROW * a, src + (int64_t)a * stride, 4);
            }
        }
    }
    for (int kk = I.Ktot; kk < Kc; ++kk) S.A[kk][threadIdx.x] = 0.f;
}

// Operand row of a tile in the in-block-symmetry mode.  The parent holds the
// canonical entries of its blocks only (a temporary written in this mode; A
// has them all), so every operand entry is read at its canonical position:
// contraction offset a joins, at parent mode q, the run of the e parent modes
// q+1 .. q+e whose blocks equal ibar (their offsets r_0 <= ... <= r_{e-1} are
// the row's i offsets at modes q .. q+e-1); sorted, the r_i < a move down one
// mode and a moves up p = #{r_i < a} modes:
//     off_q(rr) + sum_{i<p} r_i (b^{q+i} - b^{q+i+1}) + a b^{q+p}.
// Blocks that join no run (e = 0) take the plain strided copy (strides known at
// compile time for B > 0, as in s32_issue_a).
template <int B>
__device__ __noinline__ void s32_issue_a_sym(S32Stage& S, const LevelInst& I, const Tile& t, int Kc)
{
    const int g = S.sym.g[threadIdx.x];
    if (g >= 0) {
        const int R = I.R, b = B > 0 ? B : I.b, nbar = I.nbar, k = I.k;
        const int64_t bm = I.bm;
        const int pr = g / R, rr = g - pr * R;
        const float* pbase = (const float*)I.parent + (int64_t)t.parent * I.P_parent * bm;
        const int32_t* Grow = I.G + (int64_t)pr * nbar;
        const uint32_t iblk = S.sym.blk[threadIdx.x];
        int32_t io[STTSM_MAX_M];
        {
            int rem = rr;
            for (int x = 0; x < k; ++x) {
                const int q2 = rem / b;
                io[x] = rem - q2 * b;
                rem = q2;
            }
        }
        for (int ib = 0; ib < nbar; ++ib) {
            const int32_t gq = __ldg(Grow + ib);
            const int q = gq & 7;
            const float* src = pbase + (int64_t)(gq >> 3) * bm + __ldg(I.OFF + q * R + rr);
            int e = 0;
            while (q + e < k && (int)((iblk >> (8 * (q + e))) & 0xff) == ib) ++e;
            const uint32_t d0 = s32_smem(&S.A[ib * b][threadIdx.x]);
            if (e == 0 && B > 0) {
                if (q == 0) s32_copy_block<(B > 0 ? B : 1), 1>(d0, src);
                else s32_copy_q<(B > 0 ? B : 1)>(d0, src, q);
                continue;
            }
            int p = 0, corr = 0;
            for (int a = 0; a < b; ++a) {
                while (p < e && io[q + p] < a) {
                    corr += io[q + p] * (I.bpow[q + p] - I.bpow[q + p + 1]);
                    ++p;
                }
                s32_cp4(d0 + S32_KROW * a, src + corr + a * I.bpow[q + p], 4);
            }
        }
    }
    for (int kk = I.Ktot; kk < Kc; ++kk) S.A[kk][threadIdx.x] = 0.f;
}

template <typename Desc, bool SYM>
__device__ __forceinline__ void s32_issue(S32Stage& S, const Desc* insts, const LevelInst& inst0, const Tile& t,
                                          bool with_x)
{
    const LevelInst& I = insts ? level_of(insts, t.inst) : inst0;
    const int Kc = (I.Ktot + 3) & ~3;
    bool done = false;
    if constexpr (SYM) {
        if (sym_tile(t.pad0)) {
            switch (I.b) {
            case 4: s32_issue_a_sym<4>(S, I, t, Kc); break;
            case 8: s32_issue_a_sym<8>(S, I, t, Kc); break;
            case 16: s32_issue_a_sym<16>(S, I, t, Kc); break;
            default: s32_issue_a_sym<0>(S, I, t, Kc); break;
            }
            done = true;
        }
    }
    if (!done) switch (I.b) {
    case 4: s32_issue_a<4>(S, I, t, Kc); break;
    case 8: s32_issue_a<8>(S, I, t, Kc); break;
    case 16: s32_issue_a<16>(S, I, t, Kc); break;
    default: s32_issue_a<0>(S, I, t, Kc); break;
    }
    if (!with_x) return;
    switch (s32_width_class(t.ncols)) {
    case 0: s32_issue_x<8>(S, I, t, Kc); break;
    case 1: s32_issue_x<16>(S, I, t, Kc); break;
    case 2: s32_issue_x<24>(S, I, t, Kc); break;
    case 3: s32_issue_x<32>(S, I, t, Kc); break;
    case 4: s32_issue_x<48>(S, I, t, Kc); break;
    default: s32_issue_x<64>(S, I, t, Kc); break;
    }
}

// Two FP32 fused multiply-adds in one instruction: lanes (lo, hi) of d get
// d + a * x lane by lane, each rounded once like fmaf.  Pairs hold two
// consecutive output columns; a2 holds one operand entry twice.
__device__ __forceinline__ void s32_fma2(uint64_t& d, uint64_t a2, uint64_t x2)
{
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a2), "l"(x2));
}
__device__ __forceinline__ uint64_t s32_dup(float a)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
    return r;
}

// In-block symmetry: the entry of column cc of a canonical row (block prefix
// pr, offsets o of the modes != k, tie bits of the row) goes to every position
// of its child block that equals it by symmetry; the columns of the diagonal
// child (jb = u_0) beyond the offset of mode k+1 are not canonical and are
// dropped (their canonical entries are another row's).
__device__ __noinline__ void s32_sym_put(const LevelInst& I, const Tile& t, int pr, int64_t rowoff, int32_t* o,
                                         uint32_t tie, int cc, float v)
{
    const int b = I.b, k = I.k;
    const int jb = cc / b, c = cc - jb * b;
    const bool diag = k < I.m - 1 && jb == sym_u0(t.pad0);
    if (diag && c > o[k + 1]) return;
    // The range checks here never fail (every offset is a permutation of in-block
    // offsets of a block of this tile's children); they keep a broken invariant from
    // writing outside the output block.
    if (pr >= I.P_out || (k < I.m - 1 && jb > sym_u0(t.pad0))) return;
    float* blk = (float*)I.out + (((int64_t)t.child_base + jb) * I.P_out + pr) * I.bm;
    const uint32_t tb = tie | (diag ? 1u << k : 0u);
    if (tb == 0) {
        const int64_t a = rowoff + (int64_t)I.bpow[k] * c;
        if (a >= 0 && a < I.bm) blk[a] = v;
        return;
    }
    o[k] = c;
    for (int a = 0; a < I.m; ++a)
        if (o[a] < 0 || o[a] >= b) return;
    // every distinct permutation of o inside the runs of tb (m <= 5: at most 5! = 120)
    int guard = 0;
    for (;;) {
        int64_t off = 0;
        for (int a = 0; a < I.m; ++a) off += (int64_t)o[a] * I.bpow[a];
        if (off >= 0 && off < I.bm) blk[off] = v;
        if (++guard > 120) return;
        bool adv = false;
        for (int a = 0; a < I.m && !adv;) {
            int hi = a + 1;
            while (hi < I.m && ((tb >> (hi - 1)) & 1)) ++hi;
            if (hi - a > 1) adv = sym_next_perm(o, a, hi);
            a = hi;
        }
        if (!adv) break;
    }
}

// Offsets of the modes != k of row rr (row digit a is mode a below k, a + 1 above).
__device__ __forceinline__ void s32_row_digits(const LevelInst& I, int rr, int32_t* o)
{
    int rem = rr;
    const int b = I.b, lb = (b & (b - 1)) == 0 ? __ffs(b) - 1 : -1;
    for (int a = 0; a < I.m; ++a) {
        if (a == I.k) { o[a] = 0; continue; }
        const int q = lb >= 0 ? rem >> lb : rem / b;
        o[a] = rem - q * b;
        rem = q;
    }
}

// One canonical row of a tile in the in-block-symmetry mode (sym.cuh), stored
// from the registers of the thread that computed it.  For every mirror of the
// row (its offsets permuted inside each run of equal blocks, mode k apart;
// m <= 5 gives at most SYM_MAXMIR = 4! of them) the columns of the children
// other than the diagonal one go to the mirror row as in the full computation
// (4 at a time for b a power of two >= 4).  The diagonal child (jb = u_0, whose
// mode k joins the run of modes k+1 .. k+gr): a canonical column c <= o_{k+1}
// goes to the mirror row and to every position where c swaps places with the
// offset w of one mode j of that run, offset + c b^j + w (b^k - b^j) -- these
// swaps and the row's permutations give every arrangement of the run;
// columns c > o_{k+1} are another row's mirrors and are dropped.
constexpr int SYM_MAXMIR = 24;

__device__ __forceinline__ void s32_sym_diag(float* row, const LevelInst& I, const int32_t* q, int gr, int bk, int cl,
                                             float val)
{
    row[cl * bk] = val;
    for (int j = 1; j <= gr; ++j) {
        const int bj = I.bpow[I.k + j];
        row[cl * bj + q[I.k + j] * (bk - bj)] = val;
    }
}

template <int TC>
__device__ __forceinline__ void s32_sym_store_row(const float (&v)[TC], const LevelInst& I, const Tile& t, int g,
                                                  uint32_t tie, int cfirst, int nvalid)
{
    const int m = I.m, k = I.k, b = I.b, bk = I.bpow[k];
    const int pr = g / I.R, rr = g - pr * I.R;
    int32_t q[STTSM_MAX_M];
    s32_row_digits(I, rr, q);
    const int jbd = k < m - 1 ? sym_u0(t.pad0) : -1;
    int gr = 0;
    if (k < m - 1) {
        gr = 1;
        while (k + gr < m - 1 && ((tie >> (k + gr)) & 1)) ++gr;
    }
    const int ok1 = k < m - 1 ? q[k + 1] : 0;
    const int64_t child_step = (int64_t)I.P_out * I.bm;
    const float* base = (const float*)I.out + ((int64_t)t.child_base * I.P_out + pr) * I.bm;
    const bool pow2 = b >= 4 && (b & (b - 1)) == 0;
    const int lb = pow2 ? __ffs(b) - 1 : 0;
    for (int mir = 0; mir < SYM_MAXMIR; ++mir) {
        int32_t ro = 0;
        for (int x = 0; x < m; ++x)
            if (x != k) ro += q[x] * I.bpow[x];
        float* row = (float*)base + ro;
        if (pow2) {
#pragma unroll
            for (int e = 0; e < TC; e += 4) {
                if (e >= nvalid) break;
                const int cc = cfirst + e, jb = cc >> lb, c0 = cc & (b - 1);
                float* d = row + (int64_t)jb * child_step;
                if (jb != jbd) {
                    d += (int64_t)bk * c0;
                    if (bk == 1) {
                        *(float4*)d = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                    } else {
                        d[0] = v[e];
                        d[bk] = v[e + 1];
                        d[2 * bk] = v[e + 2];
                        d[3 * bk] = v[e + 3];
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (c0 + u <= ok1) s32_sym_diag(d, I, q, gr, bk, c0 + u, v[e + u]);
                }
            }
        } else {
            int jb = cfirst / b, c = cfirst - jb * b;
#pragma unroll
            for (int e = 0; e < TC; ++e) {
                if (e < nvalid) {
                    float* d = row + (int64_t)jb * child_step;
                    if (jb != jbd) d[(int64_t)bk * c] = v[e];
                    else if (c <= ok1) s32_sym_diag(d, I, q, gr, bk, c, v[e]);
                }
                if (++c == b) { c = 0; ++jb; }
            }
        }
        bool adv = false;   // next mirror: next permutation of the first run that has one
        for (int x = 0; x < m && !adv;) {
            int hi = x + 1;
            while (hi < m && ((tie >> (hi - 1)) & 1)) ++hi;
            if (hi - x > 1) adv = sym_next_perm(q, x, hi);
            x = hi;
        }
        if (!adv) break;
    }
}

// A temporary of the in-block-symmetry mode: the canonical entries of one row
// only (the next level reads those), the columns of the diagonal child past the
// offset of mode k+1 dropped.
template <int TC>
__device__ __forceinline__ void s32_sym_store_canon(const float (&v)[TC], const LevelInst& I, const Tile& t, int g,
                                                    int cfirst, int nvalid)
{
    const int b = I.b, k = I.k, bk = I.bpow[k];
    const int jbd = k < I.m - 1 ? sym_u0(t.pad0) : -1;
    const int64_t child_step = (int64_t)I.P_out * I.bm;
    const int pr = g / I.R, rr = g - pr * I.R;
    const int ok1 = (rr / bk) % b;   // offset of mode k+1 (row digit k)
    float* row = (float*)I.out + ((int64_t)t.child_base * I.P_out + pr) * I.bm + __ldg(I.OFF + k * I.R + rr);
    if (b >= 4 && (b & (b - 1)) == 0) {
        const int lb = __ffs(b) - 1;
#pragma unroll
        for (int e = 0; e < TC; e += 4) {
            if (e >= nvalid) break;
            const int cc = cfirst + e, jb = cc >> lb, c0 = cc & (b - 1);
            float* d = row + (int64_t)jb * child_step + (int64_t)bk * c0;
            if (jb != jbd) {
                if (bk == 1) {
                    *(float4*)d = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                } else {
                    d[0] = v[e];
                    d[bk] = v[e + 1];
                    d[2 * bk] = v[e + 2];
                    d[3 * bk] = v[e + 3];
                }
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (c0 + u <= ok1) d[u * bk] = v[e + u];
            }
        }
        return;
    }
    int jb = cfirst / b, c = cfirst - jb * b;
#pragma unroll
    for (int e = 0; e < TC; ++e) {
        if (e < nvalid && (jb != jbd || c <= ok1)) row[(int64_t)jb * child_step + (int64_t)bk * c] = v[e];
        if (++c == b) { c = 0; ++jb; }
    }
}

// The rows of this thread (as s32_compute_store distributes them), whose results
// it parked in its own cells of the operand stage: a separate function, so the
// full computation's register allocation does not carry these stores.  The
// call's result gets every entry (s32_sym_store_row), a temporary its canonical
// entries (s32_sym_store_canon).
template <int TC, int TR>
__device__ __noinline__ void s32_sym_store(const S32Stage& S, const LevelInst& I, const Tile& t, int r0, int part,
                                           int cfirst, int nvalid)
{
    constexpr int RSTEP = S32_ROWS / TR;
#pragma unroll 1
    for (int j = 0; j < TR; ++j) {
        const int rowi = r0 + j * RSTEP;
        const int g = S.sym.g[rowi];
        if (g < 0) continue;
        float v[TC];
#pragma unroll
        for (int e = 0; e < TC; ++e) v[e] = S.A[part * TC + e][rowi];
        if (I.sym_full) s32_sym_store_row<TC>(v, I, t, g, S.sym.tie[rowi], cfirst, nvalid);
        else s32_sym_store_canon<TC>(v, I, t, g, cfirst, nvalid);
    }
}

// This thread's canonical row of a tile in the in-block-symmetry mode.
__device__ __noinline__ void s32_sym_row(S32Stage& S, const LevelInst& I, const Tile& t)
{
    const int64_t rho = (int64_t)t.row0 + threadIdx.x;
    uint32_t tie = 0, iblk = 0;
    int64_t gg = rho < t.pad1
                     ? sym_row(S.sym.tab, I.m, I.k, I.b, I.Ktot, I.R, I.bpow, sym_pattern(t.pad0), rho, &tie, &iblk)
                     : -1;
    if (gg >= I.rows_per_parent) gg = -1;   // never (the map stays inside the parent's rows)
    S.sym.g[threadIdx.x] = (int32_t)gg;
    S.sym.tie[threadIdx.x] = tie;
    S.sym.blk[threadIdx.x] = iblk;
}

// Rows times the tile's X block, then the scatter into the children's blocks:
// output (child cb + jb, block pr) at in-block offset OFF[k][rr] + b^k c.
// A thread computes TR rows (t mod 128/TR, + 128/TR, ...) times NC/TR columns
// (part t / (128/TR)), so every X value read from shared memory feeds TR
// products; column pairs go through the two-lane FMA.
template <int NC, int TR, bool SYM>
__device__ __forceinline__ void s32_compute_store(S32Stage& S, const LevelInst& I, const Tile& t)
{
    constexpr int TC = NC / TR, RSTEP = S32_ROWS / TR;
    const int r0 = threadIdx.x % RSTEP, part = threadIdx.x / RSTEP;
    const int Kc = (I.Ktot + 3) & ~3;
    uint64_t acc[TR][TC / 2];
#pragma unroll
    for (int j = 0; j < TR; ++j)
#pragma unroll
        for (int c = 0; c < TC / 2; ++c) acc[j][c] = 0ull;
#pragma unroll 1
    for (int kk = 0; kk < Kc; kk += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const ulonglong2* xr = (const ulonglong2*)&S.X[kk + u][part * TC + s32_xshift<NC>(u)];
            uint64_t a2[TR];
#pragma unroll
            for (int j = 0; j < TR; ++j) a2[j] = s32_dup(S.A[kk + u][r0 + j * RSTEP]);
#pragma unroll
            for (int c4 = 0; c4 < TC / 4; ++c4) {
                const ulonglong2 x = xr[c4];
#pragma unroll
                for (int j = 0; j < TR; ++j) {
                    s32_fma2(acc[j][2 * c4 + 0], a2[j], x.x);
                    s32_fma2(acc[j][2 * c4 + 1], a2[j], x.y);
                }
            }
        }
    }
    const int b = I.b, bk = I.bpow[I.k];
    const int cfirst = t.col0 + part * TC;
    const int nvalid = t.ncols - part * TC;
    if constexpr (SYM) {
        if (sym_tile(t.pad0)) {
            __syncthreads();   // every thread is done reading the operand stage
    #pragma unroll
            for (int j = 0; j < TR; ++j)
    #pragma unroll
                for (int e = 0; e < TC / 2; ++e) {
                    float lo, hi;
                    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[j][e]));
                    S.A[part * TC + 2 * e][r0 + j * RSTEP] = lo;   // this thread's own cells
                    S.A[part * TC + 2 * e + 1][r0 + j * RSTEP] = hi;
                }
            s32_sym_store<TC, TR>(S, I, t, r0, part, cfirst, nvalid);
            return;
        }
    }
    if (b >= 4 && (b & (b - 1)) == 0) {
        // b a power of two >= 4: a thread's columns start on a multiple of 4 and
        // the tile's width is a multiple of b, so every group of 4 columns lies
        // inside one child block; at k = 0 it is 4 contiguous, 16-byte aligned
        // floats of the row
        const int lb = __ffs(b) - 1;
        const int64_t child_step = (int64_t)I.P_out * I.bm;
#pragma unroll
        for (int j = 0; j < TR; ++j) {
            const int g = t.row0 + r0 + j * RSTEP;
            if (g >= I.rows_per_parent) continue;
            const int pr = g / I.R, rr = g - pr * I.R;
            float* row = (float*)I.out + ((int64_t)t.child_base * I.P_out + pr) * I.bm + __ldg(I.OFF + I.k * I.R + rr);
#pragma unroll
            for (int e = 0; e < TC; e += 4) {
                if (e >= nvalid) break;
                float r4[4];
                asm("mov.b64 {%0, %1}, %2;" : "=f"(r4[0]), "=f"(r4[1]) : "l"(acc[j][e / 2]));
                asm("mov.b64 {%0, %1}, %2;" : "=f"(r4[2]), "=f"(r4[3]) : "l"(acc[j][e / 2 + 1]));
                const int cc = cfirst + e;
                float* d = row + (int64_t)(cc >> lb) * child_step + (int64_t)bk * (cc & (b - 1));
                if (bk == 1) {
                    *(float4*)d = make_float4(r4[0], r4[1], r4[2], r4[3]);
                } else {
                    d[0] = r4[0];
                    d[bk] = r4[1];
                    d[2 * bk] = r4[2];
                    d[3 * bk] = r4[3];
                }
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < TR; ++j) {
        const int g = t.row0 + r0 + j * RSTEP;
        if (g >= I.rows_per_parent) continue;
        float res[TC];
#pragma unroll
        for (int e = 0; e < TC / 2; ++e)
            asm("mov.b64 {%0, %1}, %2;" : "=f"(res[2 * e]), "=f"(res[2 * e + 1]) : "l"(acc[j][e]));
        const int pr = g / I.R, rr = g - pr * I.R;
        const int64_t rowoff = __ldg(I.OFF + I.k * I.R + rr);
        int jb = cfirst / b, c = cfirst - jb * b;
        float* dst = (float*)I.out + (((int64_t)t.child_base + jb) * I.P_out + pr) * I.bm + rowoff;
#pragma unroll
        for (int e = 0; e < TC; ++e) {
            if (e < nvalid) dst[(int64_t)bk * c] = res[e];
            if (++c == b) { c = 0; dst += I.P_out * I.bm; }
        }
    }
}

// The last level (k = 0) under the R64 precisions: one output row per thread,
// columns in chunks of at most 16; the FP32 sum over each contraction block of
// b indices is added to an FP64 sum (the cross-block accumulation of a C
// block in FP64), and C gets the FP64 sum rounded once.
template <int NC, bool SYM>
__device__ __forceinline__ void s32_compute_store_r64(const S32Stage& S, const LevelInst& I, const Tile& t)
{
    constexpr int CW = NC < 16 ? NC : 16;
    const int r = threadIdx.x;
    const bool sym = SYM && sym_tile(t.pad0);
    const int g = sym ? S.sym.g[r] : t.row0 + r;
    if (g < 0 || g >= I.rows_per_parent) return;
    const int Kc = (I.Ktot + 3) & ~3;
    const int b = I.b;
    const int pr = g / I.R, rr = g - pr * I.R;
    int32_t o[STTSM_MAX_M];
    if constexpr (SYM) {
        if (sym) s32_row_digits(I, rr, o);
    }
    float* row = (float*)I.out + ((int64_t)t.child_base * I.P_out + pr) * I.bm + __ldg(I.OFF + I.k * I.R + rr);
    const int64_t child_step = (int64_t)I.P_out * I.bm;
#pragma unroll 1
    for (int c0 = 0; c0 < NC; c0 += CW) {
        if (c0 >= t.ncols) break;
        uint64_t acc[CW / 2];
        double dacc[CW];
#pragma unroll
        for (int e = 0; e < CW / 2; ++e) acc[e] = 0ull;
#pragma unroll
        for (int e = 0; e < CW; ++e) dacc[e] = 0.0;
        int in_block = 0;
#pragma unroll 4
        for (int kk = 0; kk < Kc; ++kk) {
            const uint64_t a2 = s32_dup(S.A[kk][r]);
            const ulonglong2* xr = (const ulonglong2*)&S.X[kk][c0 + s32_xshift<NC>(kk)];
#pragma unroll
            for (int c4 = 0; c4 < CW / 4; ++c4) {
                const ulonglong2 x = xr[c4];
                s32_fma2(acc[2 * c4 + 0], a2, x.x);
                s32_fma2(acc[2 * c4 + 1], a2, x.y);
            }
            if (++in_block == b || kk == Kc - 1) {
                in_block = 0;
#pragma unroll
                for (int e = 0; e < CW / 2; ++e) {
                    float lo, hi;
                    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[e]));
                    dacc[2 * e] += (double)lo;
                    dacc[2 * e + 1] += (double)hi;
                    acc[e] = 0ull;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < CW; ++e) {
            const int cc = t.col0 + c0 + e;
            if (c0 + e >= t.ncols) break;
            if constexpr (SYM) {
                if (sym) {
                    s32_sym_put(I, t, pr, __ldg(I.OFF + I.k * I.R + rr), o, S.sym.tie[r], cc, (float)dacc[e]);
                    continue;
                }
            }
            const int jb = cc / b, c = cc - jb * b;
            row[(int64_t)jb * child_step + c] = (float)dacc[e];
        }
    }
}

// SYM: the launch has tiles in the in-block-symmetry mode (sym.cuh); the other
// instantiation carries none of that code and uses the stage without S32Sym.
template <typename Desc, bool SYM>
__global__ void __launch_bounds__(S32_ROWS, S32_CTAS_PER_SM)
level_small_f32_kernel(const Desc* __restrict__ insts, LevelInst inst0, const Tile* __restrict__ tiles, int ntiles,
                       int r64)
{
    extern __shared__ __align__(16) unsigned char s32_raw[];
    S32Stage& S = *(S32Stage*)s32_raw;
    bool tab_ready = false;   // binomial table of the symmetry mode, filled at the CTA's first such tile
    // row groups of one parent node share their X block; it stays in shared
    // memory while the CTA's next tile has the same one
    int x_inst = -1, x_col0 = -1, x_ncols = -1;
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile t = tiles[ti];
        const LevelInst& I = insts ? level_of(insts, t.inst) : inst0;
        const bool new_x = t.inst != x_inst || t.col0 != x_col0 || t.ncols != x_ncols;
        x_inst = t.inst; x_col0 = t.col0; x_ncols = t.ncols;
        if constexpr (SYM) {
            if (sym_tile(t.pad0)) {
                if (!tab_ready) {
                    sym_tab_fill(S.sym.tab, threadIdx.x, blockDim.x);
                    __syncthreads();
                    tab_ready = true;
                }
                s32_sym_row(S, I, t);   // read by the other threads after the barrier below
            }
        }
        s32_issue<Desc, SYM>(S, insts, inst0, t, new_x);
        s32_commit();
        s32_wait_all();
        __syncthreads();
        if (r64 && I.k == 0) {
            switch (s32_width_class(t.ncols)) {
            case 0: s32_compute_store_r64<8, SYM>(S, I, t); break;
            case 1: s32_compute_store_r64<16, SYM>(S, I, t); break;
            case 2: s32_compute_store_r64<24, SYM>(S, I, t); break;
            case 3: s32_compute_store_r64<32, SYM>(S, I, t); break;
            case 4: s32_compute_store_r64<48, SYM>(S, I, t); break;
            default: s32_compute_store_r64<64, SYM>(S, I, t); break;
            }
        } else switch (s32_width_class(t.ncols)) {
        case 0: s32_compute_store<8, 1, SYM>(S, I, t); break;
        case 1: s32_compute_store<16, 2, SYM>(S, I, t); break;
        case 2: s32_compute_store<24, 2, SYM>(S, I, t); break;
        case 3: s32_compute_store<32, 2, SYM>(S, I, t); break;
        case 4: s32_compute_store<48, 4, SYM>(S, I, t); break;
        default: s32_compute_store<64, 4, SYM>(S, I, t); break;
        }
        __syncthreads();
    }
}

template <typename Desc, bool SYM>
static int launch_small_f32_v(const Desc* d_insts, const LevelInst& inst0, const Tile* d_tiles, int ntiles,
                              int num_sms, cudaStream_t s, int r64)
{
    // the stage without its S32Sym part unless the launch has symmetry-mode tiles
    constexpr size_t smem = SYM ? S32_SMEM : offsetof(S32Stage, sym);
    static std::mutex mu;
    static bool attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return (int)cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 0 && dev < 64 && !attr_set[dev]) {
            const cudaError_t e = cudaFuncSetAttribute(level_small_f32_kernel<Desc, SYM>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return (int)e;
            attr_set[dev] = true;
        }
    }
    const int grid = ntiles < num_sms * S32_CTAS_PER_SM ? ntiles : num_sms * S32_CTAS_PER_SM;
    level_small_f32_kernel<Desc, SYM><<<grid, S32_ROWS, smem, s>>>(d_insts, inst0, d_tiles, ntiles, r64);
    return (int)cudaGetLastError();
}

template <typename Desc>
static int launch_small_f32(const Desc* d_insts, const LevelInst& inst0, const Tile* d_tiles, int ntiles, int num_sms,
                            cudaStream_t s, int r64, int sym)
{
    if (ntiles <= 0) return 0;
    return sym ? launch_small_f32_v<Desc, true>(d_insts, inst0, d_tiles, ntiles, num_sms, s, r64)
               : launch_small_f32_v<Desc, false>(d_insts, inst0, d_tiles, ntiles, num_sms, s, r64);
}

int launch_level_small_f32(const LevelInst& inst0, const LevelInst* d_insts, const Tile* d_tiles, int ntiles,
                           int num_sms, cudaStream_t s, int r64, int sym)
{
    return launch_small_f32<LevelInst>(d_insts, inst0, d_tiles, ntiles, num_sms, s, r64, sym);
}

int launch_level_small_f32_tc(const TcInst* d_insts, const Tile* d_tiles, int ntiles, int num_sms, cudaStream_t s,
                              int r64, int sym)
{
    LevelInst none;
    memset(&none, 0, sizeof(none));
    return launch_small_f32<TcInst>(d_insts, none, d_tiles, ntiles, num_sms, s, r64, sym);
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

