// FP32 multiply-add throughput of the device: the ALU ceiling against which the search's FFT
// arithmetic is measured (its intensity is near the FP32 ridge, so both ceilings are reported).
//
// Each thread runs 16 independent fmaf chains (enough to cover the FMA latency with a few warps
// per scheduler); 4 CTAs of 256 threads per SM keep every scheduler busy.  The chains converge to
// a fixed point (x <- x a + b with a < 1), so the values stay finite whatever the length, and a
// store guarded by an impossible value keeps the compiler from removing them.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/fmbym.h"

namespace {

__device__ float g_fma_sink;

constexpr int kChains = 16;
constexpr int kFmaThreads = 256;
constexpr int kFmaBlocksPerSm = 4;

__global__ void __launch_bounds__(kFmaThreads) k_fma_peak(int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.5e38f) g_fma_sink = s;
}

}  // namespace

extern "C" int fmbym_fp32_fma_rate(void* stream, int iters, int reps, double* fma_per_s) {
    if (iters < 1 || reps < 1 || !fma_per_s) return FMBYM_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return FMBYM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if ((e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) {
        if (t0) cudaEventDestroy(t0);
        return FMBYM_ERR_CUDA;
    }
    const dim3 grid(sms * kFmaBlocksPerSm);
    const double fmas = (double)grid.x * kFmaThreads * kChains * (double)iters;
    float best = 1e30f;
    k_fma_peak<<<grid, kFmaThreads, 0, st>>>(iters, 0.999999f, 1e-6f);   // warm-up
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(t0, st);
        k_fma_peak<<<grid, kFmaThreads, 0, st>>>(iters, 0.999999f, 1e-6f);
        cudaEventRecord(t1, st);
        if ((e = cudaEventSynchronize(t1)) != cudaSuccess) break;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, t0, t1)) == cudaSuccess) best = std::min(best, ms);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (e != cudaSuccess) return FMBYM_ERR_CUDA;
    *fma_per_s = fmas / (best * 1e-3);
    return FMBYM_OK;
}
