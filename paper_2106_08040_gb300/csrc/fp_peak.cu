// FP64 fused multiply-add throughput of the current GPU (measurement utility
// for the roofline denominator of the FP64 solver; the paper has no
// counterpart).  Every thread runs 8 independent FMA chains.
#include <cuda_runtime.h>
#include "fp_internal.h"

__global__ void __launch_bounds__(256) fp_dfma_kernel(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
           x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == 12345.678) out[blockIdx.x] = s;     // keeps the chains live
}

extern "C" int fp_peak_fp64(double* gflops) {
    if (!gflops) return FP_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FP_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double* d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * 4096) != cudaSuccess) return FP_ENOMEM;
    const int blocks = sms * 8, iters = 1 << 14;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fp_dfma_kernel<<<blocks, 256>>>(d, iters / 16, 0.999999, 1e-7);      // warm-up
    cudaEventRecord(e0);
    fp_dfma_kernel<<<blocks, 256>>>(d, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    if (err != cudaSuccess || ms <= 0.f) return FP_ECUDA;
    *gflops = 2.0 * 8.0 * (double)iters * blocks * 256 / (ms * 1e-3) / 1e9;
    return FP_OK;
}
