// FP32 FMA-pipe microbenchmark: the measured ceiling of the CGLS kernels'
// binding unit.  The convolutions (the dominant flops of every CG iteration)
// run on the FP32 FFMA pipe, whose nominal peak is SMs x 128 lanes x 2 flops
// x clock; this kernel measures what that pipe actually sustains here, with
// sixteen independent FMA chains per thread (enough to hide the FMA latency)
// on every SM.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/mirage.h"

namespace {

constexpr int PEAK_CHAINS = 16;

__global__ void __launch_bounds__(256) k_ffma_peak(float* __restrict__ out, float a, float b, int iters) {
    float acc[PEAK_CHAINS];
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) acc[j] = (float)threadIdx.x * 1e-3f + (float)j;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < PEAK_CHAINS; ++j) acc[j] = fmaf(acc[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < PEAK_CHAINS; ++j) s += acc[j];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

}  // namespace

extern "C" int mirage_measure_ffma(int device, double* tflops, double* flop_per_clk_sm) {
    if (!tflops || !flop_per_clk_sm) return MIRAGE_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return MIRAGE_ERR_CUDA;
    int sms = 0, khz = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device) != cudaSuccess || sms <= 0 || khz <= 0)
        return MIRAGE_ERR_CUDA;
    const int block = 256, grid = sms * 8, iters = 8192;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * (size_t)grid * block) != cudaSuccess) return MIRAGE_ERR_NOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MIRAGE_OK;
    float ms = 0.f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = MIRAGE_ERR_CUDA;
    if (rc == MIRAGE_OK) {
        k_ffma_peak<<<grid, block>>>(out, 0.9999f, 1e-4f, iters);  // warm-up (clocks up)
        cudaEventRecord(e0);
        k_ffma_peak<<<grid, block>>>(out, 0.9999f, 1e-4f, iters);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
            rc = MIRAGE_ERR_CUDA;
    }
    if (rc == MIRAGE_OK) {
        const double flops = 2.0 * PEAK_CHAINS * (double)iters * grid * block;
        *tflops = flops / (ms * 1e-3) / 1e12;
        *flop_per_clk_sm = flops / (ms * 1e-3) / sms / (khz * 1e3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}
