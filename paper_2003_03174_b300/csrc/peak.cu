// peak.cu -- FP32 FMA throughput of the device: the denominator of the
// follower's arithmetic roofline (measurement only; not a step of the method).
#include <cuda_runtime.h>

#include "trd_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_fma_peak(float *out, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
#pragma unroll 4
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == 1234.5f) out[threadIdx.x] = s;  // keeps the chains alive
}

}  // namespace

extern "C" int trd_measure_fp32_peak(trd_ctx_t *ctx, double *tflops)
{
    if (!ctx || !tflops) return TRD_EINVAL;
    TRD_CUDA_TRY(cudaSetDevice(ctx->device));
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TRD_CUDA_TRY(cudaMalloc(&out, 256 * sizeof(float)));
    int rc = TRD_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = TRD_ECUDA;
    const int block = 256, grid = ctx->sm_count * 8;
    float best = 1e30f;
    for (int rep = 0; rep < 5 && rc == TRD_OK; ++rep) {
        k_fma_peak<<<grid, block>>>(out, 0.9999f, 1e-4f);
        cudaEventRecord(e0);
        k_fma_peak<<<grid, block>>>(out, 0.9999f, 1e-4f);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = TRD_ECUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    if (rc == TRD_OK) {
        const double flops = 2.0 * kChains * kIters * static_cast<double>(grid) * block;
        *tflops = flops / (best * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    (void)cudaGetLastError();
    return rc;
}
