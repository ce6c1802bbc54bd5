// peak.cu -- FP32 FMA throughput of the current device (2 flops per FMA),
// the denominator of the ALU roofline of the Gram reduction.
#include <cuda_runtime.h>

#include "../../include/ntc.h"

namespace {

constexpr int kChains = 16;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_fma_burn(float* out, float seed) {
    float acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.9999f, a = 1e-7f;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fmaf(acc[c], m, a);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == 12345.678f) out[0] = s;   // keeps the chains live
}

}  // namespace

extern "C" ntc_status ntc_measure_fp32_peak(void* stream, double* tflops) {
    if (!tflops) return NTC_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NTC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NTC_ERR_CUDA;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) return NTC_ERR_OOM;
    const int blocks = sms * 8;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double best = 0.0;
    for (int rep = 0; rep < 6; ++rep) {
        cudaEventRecord(a, s);
        k_fma_burn<<<blocks, 256, 0, s>>>(out, 1.0f);
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        const double flops = 2.0 * blocks * 256.0 * kChains * (double)kIters;
        if (rep > 0 && ms > 0.f) best = flops / (ms * 1e-3) / 1e12 > best ? flops / (ms * 1e-3) / 1e12 : best;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess || best <= 0.0) return NTC_ERR_CUDA;
    *tflops = best;
    return NTC_OK;
}
