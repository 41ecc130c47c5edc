// autotune.cu — block size by measurement: every candidate b is timed on
// device buffers of its own shape, the fastest median kept and cached.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>
#include <cuda_runtime.h>
#include "sttsm.h"
#include "plan.h"
#include "launch.h"

namespace sttsm {
namespace {

// Deterministic non-zero values in [-1, 1) (an integer hash of the index; it
// only keeps the timed arithmetic away from zero operands).
template <typename T>
__global__ void fill_pattern_kernel(T* p, int64_t count, uint32_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u ^ seed;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        p[i] = (T)((double)(h & 0xFFFFu) / 32768.0 - 1.0);
    }
}

template <typename T>
int fill(void* p, int64_t count, uint32_t seed)
{
    if (count <= 0) return 0;
    fill_pattern_kernel<T><<<1024, 256>>>((T*)p, count, seed);
    return (int)cudaGetLastError();
}

std::mutex g_mu;
std::map<std::tuple<int, int, int64_t, int64_t, int, std::vector<int>>, int> g_cache;

}  // namespace
}  // namespace sttsm

extern "C" int sttsm_autotune_b_measured(int m, int64_t n, int64_t p, int prec, const int* cands, int ncand, int reps,
                                         double* times_ms)
{
    using namespace sttsm;
    if (!cands || ncand <= 0 || ncand > 64 || reps < 1 || reps > 1000) return STTSM_ERR_ARG;
    if (prec == STTSM_TF32X3) return STTSM_ERR_UNSUPPORTED;
    if (!prec_valid(prec)) return STTSM_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return STTSM_ERR_CUDA;
    const std::vector<int> cv(cands, cands + ncand);
    const auto key = std::make_tuple(dev, m, n, p, prec, cv);
    if (!times_ms) {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) return it->second;
    }
    const size_t esz = prec == STTSM_FP64 ? 8 : 4;
    int best = -1;
    double best_ms = 0.0;
    for (int c = 0; c < ncand; ++c) {
        if (times_ms) times_ms[c] = -1.0;
        const int b = cands[c];
        Shape s;
        if (b < 1 || make_shape(m, n, p, b, &s) != STTSM_OK) continue;
        const int64_t na = bcss_num_elems(m, n, b), nc = bcss_num_elems(m, p, b);
        size_t wsb = 0;
        if (na < 0 || nc < 0 || sttsm_workspace_size(m, n, p, b, prec, &wsb) != STTSM_OK) continue;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return STTSM_ERR_CUDA;
        const size_t need = (size_t)na * esz + (size_t)(p * n) * esz + (size_t)nc * esz + wsb + 4096;
        if (need > free_b / 10 * 9) continue;   // does not fit: not a candidate here
        void *A = nullptr, *X = nullptr, *C = nullptr, *W = nullptr;
        int rc = STTSM_OK;
        if (cudaMalloc(&A, (size_t)na * esz) != cudaSuccess || cudaMalloc(&X, (size_t)(p * n) * esz) != cudaSuccess ||
            cudaMalloc(&C, (size_t)nc * esz) != cudaSuccess || (wsb && cudaMalloc(&W, wsb) != cudaSuccess))
            rc = STTSM_ERR_NOMEM;
        if (rc == STTSM_OK) {
            const bool f64 = prec == STTSM_FP64;
            if ((f64 ? fill<double>(A, na, 1u) : fill<float>(A, na, 1u)) != 0 ||
                (f64 ? fill<double>(X, p * n, 2u) : fill<float>(X, p * n, 2u)) != 0)
                rc = STTSM_ERR_CUDA;
        }
        std::vector<float> ts;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (rc == STTSM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
            rc = STTSM_ERR_CUDA;
        if (rc == STTSM_OK) rc = sttsm_bcss(A, X, m, n, p, b, C, prec, W, wsb, nullptr);   // warm-up (plans, maps)
        for (int r = 0; r < reps && rc == STTSM_OK; ++r) {
            cudaEventRecord(e0, nullptr);
            rc = sttsm_bcss(A, X, m, n, p, b, C, prec, W, wsb, nullptr);
            cudaEventRecord(e1, nullptr);
            if (rc == STTSM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = STTSM_ERR_CUDA;
            float ms = 0.f;
            if (rc == STTSM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = STTSM_ERR_CUDA;
            ts.push_back(ms);
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(A); cudaFree(X); cudaFree(C); if (W) cudaFree(W);
        if (rc == STTSM_ERR_NOMEM) continue;
        if (rc != STTSM_OK) return rc;
        std::sort(ts.begin(), ts.end());
        const double med = ts[ts.size() / 2];
        if (times_ms) times_ms[c] = med;
        if (best < 0 || med < best_ms) { best = b; best_ms = med; }
    }
    if (best < 0) return STTSM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key] = best;
    return best;
}
