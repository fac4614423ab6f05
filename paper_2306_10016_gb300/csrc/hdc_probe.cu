// hdc_probe.cu -- vector FMA throughput probe (FP64 and FP32).
//
// The convolution runs on the plain FP64/FP32 pipes, not on tensor cores, so
// its arithmetic roofline is the vector FMA rate of the chip.  The probe
// runs `chains` independent FMA dependency chains per thread for `iters`
// iterations; one FMA counts as 2 flops.  The caller times the launch with
// CUDA events and divides 2 * chains * iters * threads * blocks by it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hdc.h"

#define HDC_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

template <typename T, int CH>
__global__ void k_fma_probe(T* out, int64_t iters, T x, T y)
{
    T a[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) a[c] = fma(a[c], x, y);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += a[c];
    if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s; // never true; keeps the chains live
}

} // namespace

HDC_EXPORT int hdc_probe_fma(int dtype, int64_t iters, int blocks, int threads, void* out, void* stream,
                             double* flops)
{
    if (iters < 1 || blocks < 1 || threads < 1 || threads > 1024 || !out) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    constexpr int CH = 8;
    if (dtype == HDC_C128)
        k_fma_probe<double, CH><<<blocks, threads, 0, st>>>((double*)out, iters, 0.999999, 1e-7);
    else if (dtype == HDC_C64)
        k_fma_probe<float, CH><<<blocks, threads, 0, st>>>((float*)out, iters, 0.999999f, 1e-7f);
    else
        return HDC_ERR_DTYPE;
    if (flops) *flops = 2.0 * CH * (double)iters * (double)threads * (double)blocks;
    return cudaGetLastError() == cudaSuccess ? HDC_OK : HDC_ERR_CUDA;
}
