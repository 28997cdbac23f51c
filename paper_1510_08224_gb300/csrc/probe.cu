// Measurement helper with no counterpart in the paper: the device's FP64
// fused multiply-add rate, the ceiling of the FP64-storage step kernel (whose
// 108 FP64 instructions per cell bind it, not HBM). Each thread runs eight
// independent DFMA chains x <- x a + b (a, b chosen so x stays near 1) on a
// grid of eight 256-thread blocks per SM; the best of five CUDA-event timed
// launches gives DFMA instructions per second (2 flops each).
#include <cuda_runtime.h>

#include <cmath>

#include "nomrt_internal.h"
#include "nomrt_lbm.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kIters = 2048;

// Written only if the chains' sum were -1, which never happens (every x stays
// near 1); the store keeps the compiler from dropping the chains.
__device__ double g_dfma_sink;

__global__ void __launch_bounds__(kThreads) k_dfma_rate(int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0) g_dfma_sink = s;
}

lbm_status probe_fail(lbm_status st, const char *msg) {
    nomrt::set_thread_error(msg);
    return st;
}

}  // namespace

extern "C" lbm_status lbm_probe_fp64_rate(void *cuda_stream, double *dfma_per_s) {
    if (!dfma_per_s) return probe_fail(LBM_EINVAL, "dfma_per_s is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = 8 * (sms > 0 ? sms : 1);
    const double a = 1.0 - 1.0 / 1024, b = 1.0 / 1024;  // fixed point x = 1
    float best = INFINITY;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {  // the first launch is a warm-up
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) k_dfma_rate<<<blocks, kThreads, 0, s>>>(kIters, a, b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return probe_fail(LBM_ECUDA, cudaGetErrorString(e));
    const double fmas = (double)blocks * kThreads * kIters * kChains;
    *dfma_per_s = fmas / (best * 1e-3);
    return LBM_OK;
}
