// Measured FP32 multiply-add rate of the current GPU: the roofline denominator of the kernels that
// are bound by the FP32 pipe (spread and interpolation do ~77 flop per algorithmic byte, far above
// the pipe's balance against HBM). Each thread runs eight independent chains of paired FMAs
// (fma.rn.f32x2), so the pipe, not latency, limits the rate.
#include <cuda_runtime.h>

#include <algorithm>

#include "anova_internal.h"
#include "kernels_common.cuh"

namespace anova {
namespace {

constexpr int kPeakChains = 8;
constexpr int kPeakIters = 4096;

__global__ void __launch_bounds__(256) k_fma_peak(float seed, float *sink) {
    f32x2 acc[kPeakChains];
    const f32x2 m = make_float2(0.999999f, 1.000001f), c = make_float2(1e-7f, -1e-7f);
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) acc[k] = make_float2(seed + threadIdx.x + k, seed - k);
#pragma unroll 4
    for (int it = 0; it < kPeakIters; ++it)
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) acc[k] = fma2(acc[k], m, c);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += acc[k].x + acc[k].y;
    if (s == 1234.5f) sink[0] = s;  // never true for these inputs; keeps the chains live
}

}  // namespace
}  // namespace anova

using namespace anova;

extern "C" anova_status anova_measure_fp32_peak(double *tflops) {
    if (!tflops) return fail(ANOVA_ERR_INVALID_ARG, "tflops is NULL");
    int dev = 0, sms = 0;
    ANOVA_CUDA_TRY(cudaGetDevice(&dev));
    ANOVA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t st = nullptr;
    struct Cleanup {
        float *&sink;
        cudaEvent_t &a, &b;
        cudaStream_t &st;
        ~Cleanup() {
            if (st) cudaStreamSynchronize(st);
            if (sink) cudaFree(sink);
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
            if (st) cudaStreamDestroy(st);
        }
    } cleanup{sink, a, b, st};
    ANOVA_CUDA_TRY(cudaMalloc(&sink, sizeof(float)));
    ANOVA_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ANOVA_CUDA_TRY(cudaEventCreate(&a));
    ANOVA_CUDA_TRY(cudaEventCreate(&b));
    const int blocks = sms * 8;
    k_fma_peak<<<blocks, 256, 0, st>>>(1.0f, sink);  // warm-up
    ANOVA_CUDA_TRY(cudaGetLastError());
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        ANOVA_CUDA_TRY(cudaEventRecord(a, st));
        k_fma_peak<<<blocks, 256, 0, st>>>(1.0f + rep, sink);
        ANOVA_CUDA_TRY(cudaEventRecord(b, st));
        ANOVA_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.0f;
        ANOVA_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        best = std::min(best, ms);
    }
    const double flops = 2.0 * 2.0 * kPeakChains * (double)kPeakIters * 256.0 * blocks;  // 2 lanes x FMA
    *tflops = flops / (best * 1e-3) / 1e12;
    return ANOVA_OK;
}
