// Instantiation of the fused stream-and-collide kernels for f64 population storage.
#include "launchers.cuh"

namespace nomrt {
const Launchers &launchers_f64() {
    static const Launchers L = make_launchers<double>();
    return L;
}
}  // namespace nomrt

namespace nomrt {

// One block sums partials[kRedBlocks][width] column by column in a fixed
// order, so repeated reductions of the same data give the same bits.
__global__ void __launch_bounds__(kRedThreads) k_reduce_partials(const double *partials, int width, double *out) {
    __shared__ double sh[kRedThreads];
    for (int k = 0; k < width; ++k) {
        double a = 0.0;
        for (int b = threadIdx.x; b < kRedBlocks; b += kRedThreads) a += partials[b * width + k];
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int s = kRedThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

cudaError_t reduce_partials(const double *partials, int width, double *out, cudaStream_t st) {
    k_reduce_partials<<<1, kRedThreads, 0, st>>>(partials, width, out);
    return cudaGetLastError();
}

}  // namespace nomrt
