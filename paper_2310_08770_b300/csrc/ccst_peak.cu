// FP32 FMA throughput of the device: the denominator of the tracking kernel's roofline.
//
// The hot path's dense work (the upsampled-DFT contraction of Sec. III and the FFTs of
// Eq. (4)) must keep FP32-level accuracy, so its roofline is the rate of the plain FP32
// FMA pipes. This file measures that rate with a kernel of independent FMA chains that
// fill every SM, and reports the nominal figure from the device's own attributes beside it
// (SMs x 128 FP32 lanes x 2 flop x the reported peak clock).
#include <cuda_runtime.h>

#include <cstdio>

#include "ccst.h"

namespace {

constexpr int kChains = 8;        // independent chains per thread (covers the FMA latency)
constexpr int kUnroll = 16;       // FMAs per chain per loop trip
constexpr int kPeakThreads = 512;
constexpr int kPeakBlocksPerSm = 4;   // 2048 threads: the SM's full thread capacity

__device__ float g_fma_sink;

__global__ void __launch_bounds__(kPeakThreads) fma_chains(int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + 1e-7f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    // data-dependent store the compiler cannot drop; it happens for no realistic input
    if (s == -1.0f) g_fma_sink = s;
}

}  // namespace

extern "C" int ccst_fp32_fma_peak(void* stream_v, int iters, double* tflops, double* nominal_tflops) {
    if (!tflops || !nominal_tflops || iters < 1) return CCST_E_INVALID;
    cudaStream_t stream = (cudaStream_t)stream_v;
    int dev = 0, sms = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess)
        return CCST_E_CUDA;
    *nominal_tflops = (double)sms * 128.0 * 2.0 * (double)khz * 1e3 / 1e12;
    const int grid = sms * kPeakBlocksPerSm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return CCST_E_CUDA;
    }
    // b just below 1 and c small keep every chain finite and normal for any iters
    const float b = 0.99999994f, c = 1e-7f;
    double best_ms = 1e300;
    int rc = CCST_OK;
    for (int rep = 0; rep < 4 && rc == CCST_OK; ++rep) {          // rep 0 is the warm-up
        if (cudaEventRecord(e0, stream) != cudaSuccess) { rc = CCST_E_CUDA; break; }
        fma_chains<<<grid, kPeakThreads, 0, stream>>>(iters, b, c);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, stream) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess) { rc = CCST_E_CUDA; break; }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = CCST_E_CUDA; break; }
        if (rep > 0 && ms < best_ms) best_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double flop = (double)grid * kPeakThreads * (double)iters * kUnroll * kChains * 2.0;
    *tflops = flop / (best_ms * 1e-3) / 1e12;
    return CCST_OK;
}
