// lbm_residual_fields_noalloc: the steady-state residual reduction for callers
// that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not an option -- inside a
// serving loop whose device memory is fully pre-budgeted by admission control,
// inside another framework that owns the allocator and forbids side
// allocations, or on a hot path that must not hit the driver's allocator (an
// allocation can synchronise the device). Such a caller holds its macroscopic
// fields in its own device buffers and only wants the reduction.
//
// The block partial sums of the reduction live in a file-scope device array of
// fixed size (kNaScratchDoubles doubles, about 164 KB). Every GPU that loads
// this library holds that array until the process exits. Every call on a
// device shares it and it keeps the last call's contents; each call writes all
// the partials it later reads, so nothing needs clearing, but calls whose
// kernels overlap on the GPU (different streams, no ordering) race on it.
//
// The array's device address is looked up with cudaGetSymbolAddress at the
// first call on a device and cached with the id of the CUDA context that was
// current then. A later call in another context of that device (after
// cudaDeviceReset, or a primary-context reset by a host framework, which
// reloads the module and may move the array) sees a different id and looks
// the address up again.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "nomrt_internal.h"
#include "nomrt_lbm.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 16;                                   // cells per thread
constexpr int kNaCellsPerBlock = kNaThreads * kNaItems;        // 4096
constexpr int kNaMaxBlocks = 4096;
constexpr long long kNaMaxCells = (long long)kNaMaxBlocks * kNaCellsPerBlock;  // 16,777,216
constexpr int kNaWidth = 5;  // |du|^2, |u|^2, dT^2, T^2, non-finite count
constexpr int kNaScratchDoubles = kNaMaxBlocks * kNaWidth + 8;
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) double g_na_scratch[kNaScratchDoubles];

// Device address of g_na_scratch per device, with the id of the context it was
// looked up in (0: not yet looked up).
double *g_na_ptr[kNaMaxDevices] = {};
unsigned long long g_na_ctx[kNaMaxDevices] = {};
std::mutex g_na_mutex;

__global__ void __launch_bounds__(kNaThreads)
    k_na_partials(const double *ux, const double *uy, const double *T, const double *uxp, const double *uyp,
                  const double *Tp, const uint8_t *solid, long long n, double *partials) {
    double v[kNaWidth] = {0, 0, 0, 0, 0};
    const long long base = (long long)blockIdx.x * kNaCellsPerBlock;
#pragma unroll 4
    for (int k = 0; k < kNaItems; ++k) {
        const long long c = base + (long long)k * kNaThreads + threadIdx.x;
        if (c >= n) break;
        if (solid && solid[c]) continue;
        const double a = ux[c], b = uy[c], t = T[c];
        const double da = a - uxp[c], db = b - uyp[c], dt = t - Tp[c];
        v[0] += da * da + db * db;
        v[1] += a * a + b * b;
        v[2] += dt * dt;
        v[3] += t * t;
        if (!isfinite(a) || !isfinite(b) || !isfinite(t) || !isfinite(da) || !isfinite(db) || !isfinite(dt))
            v[4] += 1.0;
    }
    __shared__ double sh[kNaThreads / 32][kNaWidth];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kNaWidth; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < kNaWidth; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int k = 0; k < kNaWidth; ++k) {
            double a = lane < kNaThreads / 32 ? sh[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) partials[blockIdx.x * kNaWidth + k] = a;
        }
    }
}

// One block sums the first `nblocks` partials in a fixed order into out[kNaWidth].
__global__ void __launch_bounds__(kNaThreads) k_na_final(const double *partials, int nblocks, double *out) {
    __shared__ double sh[kNaThreads];
    for (int k = 0; k < kNaWidth; ++k) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += kNaThreads) a += partials[b * kNaWidth + k];
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int s = kNaThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

// Errors go to the calling thread's message that lbm_last_error(NULL) returns.
lbm_status na_fail(lbm_status st, const char *msg) {
    nomrt::set_thread_error(msg);
    return st;
}

// Id of the calling thread's current CUDA context (driver entry points looked
// up through the runtime, so the library needs no link to libcuda).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

lbm_status na_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa = cudaDriverEntryPointSymbolNotFound, qb = qa;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
        if (e != cudaSuccess || qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b) {
            cudaGetLastError();
            return na_fail(LBM_ECUDA, "the driver does not provide cuCtxGetCurrent / cuCtxGetId");
        }
        get_current = reinterpret_cast<CtxGetCurrentFn>(a);
        get_id = reinterpret_cast<CtxGetIdFn>(b);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS)
        return na_fail(LBM_ECUDA, "no current CUDA context");
    return LBM_OK;
}

// The scratch array's device address on the current device: looked up at the
// first call on the device (set-up), and again whenever the device's current
// context is not the one the cached address belongs to.
lbm_status na_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(LBM_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kNaMaxDevices) return na_fail(LBM_EINVAL, "device index out of range");
    // binds the device's primary context to this thread (initialising it if needed) before the
    // driver is asked for the current context
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) return na_fail(LBM_ECUDA, cudaGetErrorString(e));
    unsigned long long ctx = 0;
    lbm_status st = na_context_id(&ctx);
    if (st != LBM_OK) return st;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev] || g_na_ctx[dev] != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return na_fail(LBM_ECUDA, "cudaGetSymbolAddress of the residual scratch failed");
        }
        g_na_ptr[dev] = static_cast<double *>(p);
        g_na_ctx[dev] = ctx;
    }
    *out = g_na_ptr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_residual_fields_noalloc(const double *ux, const double *uy, const double *T, const double *ux_prev,
                                       const double *uy_prev, const double *T_prev, const uint8_t *solid,
                                       int64_t n, void *cuda_stream, double *r) {
    if (!r) return na_fail(LBM_EINVAL, "r is NULL");
    if (n < 0) return na_fail(LBM_EINVAL, "n must be >= 0");
    if (n > kNaMaxCells)
        return na_fail(LBM_EINVAL,
                       "n exceeds the 16,777,216 cells the fixed residual scratch can reduce; use lbm_residual");
    if (n > 0 && (!ux || !uy || !T || !ux_prev || !uy_prev || !T_prev))
        return na_fail(LBM_EINVAL, "a field pointer is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the call reads its result back and waits for the stream: never legal inside a capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(s, &cap);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return na_fail(LBM_ECUDA, cudaGetErrorString(ce));
    }
    if (cap != cudaStreamCaptureStatusNone)
        return na_fail(LBM_EINVAL, "lbm_residual_fields_noalloc must not be called on a stream that is being captured");
    double *scratch = nullptr;
    lbm_status st = na_scratch(&scratch);
    if (st != LBM_OK) return st;
    double sums[kNaWidth] = {0, 0, 0, 0, 0};
    if (n > 0) {
        const int nblocks = (int)((n + kNaCellsPerBlock - 1) / kNaCellsPerBlock);
        double *partials = scratch;
        double *result = scratch + kNaMaxBlocks * kNaWidth;
        k_na_partials<<<nblocks, kNaThreads, 0, s>>>(ux, uy, T, ux_prev, uy_prev, T_prev, solid, (long long)n,
                                                     partials);
        k_na_final<<<1, kNaThreads, 0, s>>>(partials, nblocks, result);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return na_fail(LBM_ECUDA, cudaGetErrorString(e));
        e = cudaMemcpyAsync(sums, result, sizeof sums, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return na_fail(LBM_ECUDA, cudaGetErrorString(e));
    }
    if (sums[4] > 0.0 || !std::isfinite(sums[0]) || !std::isfinite(sums[1]) || !std::isfinite(sums[2]) ||
        !std::isfinite(sums[3])) {
        *r = NAN;
        return na_fail(LBM_EDIVERGED, "non-finite velocity or temperature");
    }
    const double du = std::sqrt(sums[1]), dT = std::sqrt(sums[3]);
    const double Ru = std::sqrt(sums[0]) / (du > 1e-300 ? du : 1e-300);
    const double RT = std::sqrt(sums[2]) / (dT > 1e-300 ? dT : 1e-300);
    *r = Ru > RT ? Ru : RT;
    return LBM_OK;
}

}  // extern "C"
