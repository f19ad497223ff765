// Measured FP32 roof of the GPU the library runs on: a grid of independent
// fused multiply-add chains (eight per thread, several blocks per SM) timed
// with CUDA events.  Measurement plumbing for the roofline of the bond
// kernel; it computes nothing of the method.
#include <cuda_runtime.h>

#include "ppm_internal.cuh"

namespace {

__device__ float g_peak_sink;   // keeps the chains live; written only if their sum is exactly 0.5

constexpr int kChains = 8, kUnroll = 16, kThreads = 256, kBlocksPerSM = 8;

__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int q = 0; q < kChains; q++) x[q] = (float)threadIdx.x * 1e-3f + (float)q;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int r = 0; r < kUnroll; r++)
#pragma unroll
            for (int q = 0; q < kChains; q++) x[q] = __fmaf_rn(x[q], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < kChains; q++) s += x[q];
    if (s == 0.5f) g_peak_sink = s;
}

}  // namespace

extern "C" int ppm_measure_fp32_peak(void* cuda_stream, double* tflops) {
    if (!tflops) return PPM_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return PPM_ECUDA;
    const int blocks = sms * kBlocksPerSM, iters = 2048;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return PPM_ECUDA;
    }
    int rc = PPM_OK;
    float best = 0.0f;
    k_fma_chains<<<blocks, kThreads, 0, st>>>(iters / 8, 0.999f, 1e-3f);      // warm-up
    for (int rep = 0; rep < 3 && rc == PPM_OK; rep++) {
        float ms = 0.0f;
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = PPM_ECUDA; break; }
        k_fma_chains<<<blocks, kThreads, 0, st>>>(iters, 0.999f, 1e-3f);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = PPM_ECUDA;
            break;
        }
        if (ms > 0.0f && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double flops = 2.0 * (double)blocks * kThreads * iters * kUnroll * kChains;
    *tflops = flops / (best * 1e-3) / 1e12;
    return PPM_OK;
}
