// Launchers of every kernel for one storage type, and the Launchers table.
// Included once per kernel translation unit.
#pragma once

#include "nomrt_kernels.cuh"
#include "step_tma.cuh"

namespace nomrt {


inline dim3 step_block() { return dim3(128, 2); }

// Stages of the TMA pipeline per storage type: about 88 KB of shared memory per
// CTA, so two CTAs fit on an SM.
template <typename S>
struct TmaStages;
template <>
struct TmaStages<float> {
    static constexpr int value = 3;
};
template <>
struct TmaStages<__half> {
    static constexpr int value = 6;
};

template <typename S>
constexpr size_t tma_smem_bytes() {
    constexpr int HALO = 16 / (int)sizeof(S);
    return (size_t)TmaStages<S>::value * kQ * (kTmaW + 2 * HALO) * sizeof(S) + 8 * TmaStages<S>::value;
}

// Persistent grid of the TMA kernel: resident CTAs per SM x SMs, computed once
// per device.
template <typename S>
cudaError_t tma_grid(int *blocks) {
    static int cached_dev = -1, cached_blocks = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != cached_dev) {
        auto kern = k_step_tma<S, TmaStages<S>::value>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes<S>());
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTmaThreads, tma_smem_bytes<S>());
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        cached_blocks = (per_sm > 0 ? per_sm : 1) * sms;
        cached_dev = dev;
    }
    *blocks = cached_blocks;
    return cudaSuccess;
}

template <typename S>
cudaError_t launch_step(const KParams &p, int src, cudaStream_t st) {
    using C = typename Store<S>::C;
    int variant = p.variant;
    if constexpr (Store<S>::kShifted) {
        if (variant == kStepAuto) variant = kStepVec4;
    } else {
        variant = kStepScalar;
    }
    if constexpr (Store<S>::kShifted) {
        if (variant == kStepTma) {
            TmaUnits U;
            U.y_lo = p.py ? 0 : 1;
            U.nrows = p.py ? p.ny : p.ny - 2;
            U.nseg = (p.pitch + kTmaW - 1) / kTmaW;
            U.total = U.nrows > 0 ? U.nrows * U.nseg : 0;
            if (U.total == 0) return cudaSuccess;
            int blocks = 0;
            cudaError_t e = tma_grid<S>(&blocks);
            if (e != cudaSuccess) return e;
            if (blocks > U.total) blocks = U.total;
            k_step_tma<S, TmaStages<S>::value><<<blocks, kTmaThreads, tma_smem_bytes<S>(), st>>>(
                make_planes<S>(p, src), make_geom(p), make_rates<float>(p), U, p.status);
            return cudaGetLastError();
        }
        if (variant == kStepVec4) {
            // four cells per thread, 128 threads per block, one row per block row
            const int threads_x = p.pitch / 4;
            const dim3 grid((threads_x + 127) / 128, p.ny < 65535 ? p.ny : 65535);
            k_step4<S><<<grid, 128, 0, st>>>(make_planes<S>(p, src), make_geom(p), make_rates<float>(p));
            return cudaGetLastError();
        }
    }
    const dim3 b = step_block();
    const int gy = (p.ny + (int)b.y - 1) / (int)b.y;
    const dim3 grid((p.nx + b.x - 1) / b.x, gy < 65535 ? gy : 65535);
    k_step<S><<<grid, b, 0, st>>>(make_planes<S>(p, src), make_geom(p), make_rates<C>(p));
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_init_rows(const KParams &p, int buf, int r0, int r1, const double *T, cudaStream_t st) {
    const dim3 grid((p.pitch + 127) / 128, r1 - r0);
    k_init_rows<S><<<grid, 128, 0, st>>>(make_planes<S>(p, buf), make_geom(p), r0, r1, T, p.T_ref, p.varpi,
                                         Store<S>::kShifted ? 1 : 0);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_macro_rows(const KParams &p, int buf, int r0, int r1, double *out, cudaStream_t st) {
    using C = typename Store<S>::C;
    const dim3 grid((p.nx + 127) / 128, r1 - r0);
    k_macro_rows<S><<<grid, 128, 0, st>>>(make_planes<S>(p, buf), make_geom(p), make_rates<C>(p), r0, r1,
                                          p.rho_ref, p.T_ref, out);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_export_rows(const KParams &p, int buf, int r0, int r1, double *out, cudaStream_t st) {
    const dim3 grid((p.nx + 127) / 128, r1 - r0);
    k_export_rows<S><<<grid, 128, 0, st>>>(make_planes<S>(p, buf), make_geom(p), r0, r1, p.rho_ref, p.T_ref,
                                           p.varpi, out);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_import_rows(const KParams &p, int buf, int r0, int r1, const double *in, int which,
                               cudaStream_t st) {
    const dim3 grid((p.nx + 127) / 128, r1 - r0);
    k_import_rows<S><<<grid, 128, 0, st>>>(make_planes<S>(p, buf), make_geom(p), r0, r1, p.rho_ref, p.T_ref,
                                           p.varpi, in, which);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_nusselt(const KParams &p, int buf, int side, double L, double dT, double *partials,
                           cudaStream_t st) {
    k_nusselt<S><<<kRedBlocks, kRedThreads, 0, st>>>(make_planes<S>(p, buf), make_geom(p), side, L, dT, p.T_ref,
                                                    partials);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_residual(const KParams &p, int buf, double *snap, int have_snap, double *partials,
                            cudaStream_t st) {
    using C = typename Store<S>::C;
    k_residual<S><<<kRedBlocks, kRedThreads, 0, st>>>(make_planes<S>(p, buf), make_geom(p), make_rates<C>(p),
                                                     p.T_ref, snap, p.plane, have_snap, partials);
    return cudaGetLastError();
}

template <typename S>
Launchers make_launchers() {
    Launchers L;
    L.step = &launch_step<S>;
    L.init_rows = &launch_init_rows<S>;
    L.macro_rows = &launch_macro_rows<S>;
    L.export_rows = &launch_export_rows<S>;
    L.import_rows = &launch_import_rows<S>;
    L.nusselt = &launch_nusselt<S>;
    L.residual = &launch_residual<S>;
    return L;
}

}  // namespace nomrt
