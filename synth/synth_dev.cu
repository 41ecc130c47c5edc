// synth_dev.cu — device side of the seeded input generators (see synth.h).
// Fills a dense symmetric Uniform(-1,1) tensor in dimensional order directly
// in device memory, bit-identical to synth_sym_uniform_dense_f64 on the host.
#include <cuda_runtime.h>
#include <stdint.h>
#include "synth.h"

template <typename T>
__global__ void synth_fill_kernel(T* out, int m, int64_t n, uint64_t seed, int64_t total)
{
    for (int64_t lin = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; lin < total;
         lin += (int64_t)gridDim.x * blockDim.x) {
        int64_t idx[16];
        int64_t r = lin;
        for (int a = 0; a < m; ++a) { idx[a] = r % n; r /= n; }
        out[lin] = (T)synth_uniform_pm1(seed, synth_sym_key(idx, m, n));
    }
}

// dtype: 0 = FP64, 1 = FP32. Returns 0 or a cudaError_t value.
extern "C" int synth_dev_sym_uniform_dense(void* out, int m, int64_t n, uint64_t seed, int dtype, void* stream)
{
    if (m < 1 || m > 16 || n < 1) return (int)cudaErrorInvalidValue;
    int64_t total = 1;
    for (int a = 0; a < m; ++a) total *= n;
    int grid = (int)((total + 255) / 256);
    if (grid > 152 * 32) grid = 152 * 32;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == 0) synth_fill_kernel<double><<<grid, 256, 0, s>>>((double*)out, m, n, seed, total);
    else synth_fill_kernel<float><<<grid, 256, 0, s>>>((float*)out, m, n, seed, total);
    return (int)cudaGetLastError();
}
