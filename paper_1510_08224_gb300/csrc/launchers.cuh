// Launchers of every kernel for one storage type, and the Launchers table.
// Included once per kernel translation unit.
#pragma once

#include <atomic>

#include "nomrt_kernels.cuh"
#include "step8.cuh"
#include "step_tma.cuh"

namespace nomrt {


inline dim3 step_block() { return dim3(128, 2); }

// TMA kernel shapes selectable at run time (lbm_set_step_kernel config index):
// cells per thread N, threads per CTA T, stages, CTAs per SM asked of ptxas.
// Stage counts keep each CTA's shared memory near 60 or 90 KB.
constexpr int kTmaConfigs = 5;

template <typename S>
struct TmaShape;
// FP32: a 512-cell stage is 14 x 520 x 4 B = 29 KB, a 256-cell stage 14.8 KB
template <>
struct TmaShape<float> {
    static constexpr int N[kTmaConfigs] = {4, 2, 1, 1, 2};
    static constexpr int T[kTmaConfigs] = {128, 256, 512, 256, 128};
    static constexpr int ST[kTmaConfigs] = {3, 3, 3, 4, 5};
    static constexpr int MB[kTmaConfigs] = {2, 2, 2, 3, 3};
};
// FP16: half the bytes per stage, so twice the stages
template <>
struct TmaShape<__half> {
    static constexpr int N[kTmaConfigs] = {4, 2, 1, 1, 2};
    static constexpr int T[kTmaConfigs] = {128, 256, 512, 256, 128};
    static constexpr int ST[kTmaConfigs] = {6, 6, 6, 8, 10};
    static constexpr int MB[kTmaConfigs] = {2, 2, 2, 3, 3};
};

template <typename S, int N, int T, int STAGES>
constexpr size_t tma_smem_bytes() {
    constexpr int HALO = 16 / (int)sizeof(S);
    return (size_t)STAGES * kQ * (N * T + 2 * HALO) * sizeof(S) + 8 * STAGES;
}

template <typename S, int N, int T, int STAGES, int MB>
cudaError_t launch_tma_shape(const KParams &p, int src, cudaStream_t st) {
    constexpr int W = N * T;
    constexpr size_t smem = tma_smem_bytes<S, N, T, STAGES>();
    auto kern = k_step_tma<S, N, T, STAGES, MB>;
    // persistent grid: resident CTAs per SM x SMs, computed once per device (0: not yet;
    // threads that race here compute and store the same value)
    static std::atomic<int> cached[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int cached_blocks = cached[dev].load(std::memory_order_acquire);
    if (cached_blocks == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        cached_blocks = (per_sm > 0 ? per_sm : 1) * sms;
        cached[dev].store(cached_blocks, std::memory_order_release);
    }
    TmaUnits U;
    U.y_lo = p.py ? 0 : 1;
    U.nrows = p.py ? p.ny : p.ny - 2;
    U.nseg = (p.pitch + W - 1) / W;
    U.total = U.nrows > 0 ? U.nrows * U.nseg : 0;
    if (U.total == 0) return cudaSuccess;
    const int blocks = cached_blocks < U.total ? cached_blocks : U.total;
    kern<<<blocks, T, smem, st>>>(make_planes<S>(p, src), make_geom(p), make_rates<float>(p), U, p.status);
    return cudaGetLastError();
}

template <typename S, int C>
cudaError_t launch_tma_cfg(const KParams &p, int src, cudaStream_t st) {
    using Sh = TmaShape<S>;
    return launch_tma_shape<S, Sh::N[C], Sh::T[C], Sh::ST[C], Sh::MB[C]>(p, src, st);
}

template <typename S>
cudaError_t launch_tma(const KParams &p, int src, cudaStream_t st) {
    switch (p.config) {
        case 1: return launch_tma_cfg<S, 1>(p, src, st);
        case 2: return launch_tma_cfg<S, 2>(p, src, st);
        case 3: return launch_tma_cfg<S, 3>(p, src, st);
        case 4: return launch_tma_cfg<S, 4>(p, src, st);
        default: return launch_tma_cfg<S, 0>(p, src, st);
    }
}

template <typename S>
cudaError_t launch_step_variant(const KParams &p, int variant, int src, cudaStream_t st);

template <typename S>
cudaError_t launch_nee(const KParams &p, int src, cudaStream_t st) {
    using C = typename Store<S>::C;
    if (p.n_nee == 0) return cudaSuccess;
    const dim3 grid((p.n_nee + 127) / 128);
    const Planes<S> pl = make_planes<S>(p, src);
    const Geom g = make_geom(p);
    const RatesC<C> r = make_rates<C>(p);
    if (p.tq == 9) {
        if (p.bgk) k_nee<S, 9, true><<<grid, 128, 0, st>>>(pl, g, r, p.nee, p.n_nee);
        else k_nee<S, 9, false><<<grid, 128, 0, st>>>(pl, g, r, p.nee, p.n_nee);
    } else {
        if (p.bgk) k_nee<S, 5, true><<<grid, 128, 0, st>>>(pl, g, r, p.nee, p.n_nee);
        else k_nee<S, 5, false><<<grid, 128, 0, st>>>(pl, g, r, p.nee, p.n_nee);
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_step_main(const KParams &p, int src, cudaStream_t st);

// One step: the main kernel over fluid cells, then the boundary nodes of NEE walls.
template <typename S>
cudaError_t launch_step(const KParams &p, int src, cudaStream_t st) {
    cudaError_t e = launch_step_main<S>(p, src, st);
    if (e != cudaSuccess) return e;
    return launch_nee<S>(p, src, st);
}

template <typename S>
cudaError_t launch_step_main(const KParams &p, int src, cudaStream_t st) {
    int variant = p.variant;
    KParams q = p;
    if constexpr (Store<S>::kShifted) {
        // fastest measured on GB300 (4096 x 2048 cells): four cells per thread
        if (variant == kStepAuto) {
            variant = kStepVec4;
            // VEC4 configs measured fastest on GB300 (4096 x 2048 cells, with the L2
            // prefetch of the link map): D2Q5 5 resident blocks per SM (4 for BGK in FP32);
            // the D2Q9 temperature model, which keeps nine more values per cell in
            // registers, 4
            if (p.tq == 9) q.config = 0;
            else q.config = (p.bgk && sizeof(S) == 4) ? 0 : 1;
            // FP32 MRT D2Q5 rows that are not a multiple of 512 cells: the per-warp form,
            // which leaves no warp of a block idle at a row's end (600 x 600: 0.77 -> 0.82
            // of the copy peak, 1100 x 900: 0.88 -> 0.91); in FP16 its per-warp prefetches
            // measured slower (4096 x 2048: 0.78 against 0.96)
            if (sizeof(S) == 4 && p.tq == 5 && !p.bgk && p.pitch % 512 != 0) variant = kStepVec4w;
        }
    } else {
        variant = kStepScalar;
    }
    return launch_step_variant<S>(q, variant, src, st);
}

// SMs of the current device, read once per device (0 if it cannot be read).
inline int device_sms() {
    constexpr int kDevices = 16;
    static std::atomic<int> sms[kDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) return 0;
    int n = sms[dev].load(std::memory_order_relaxed);
    if (n == 0 && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
        sms[dev].store(n, std::memory_order_relaxed);
    return n;
}

// A step of the four-cell kernel, as a programmatic dependent of the launch before
// it on the stream where its grid spans more than one wave of resident blocks
// (MINB per SM): its blocks become resident while the previous step's last blocks
// finish and wait there (griddepcontrol.wait) for that grid's completion, which
// hides the launch latency between back-to-back steps. Measured on GB300: 4096 x
// 2048 +0.2 %, a 1024^2 cavity +1.8 % (FP16); grids of under one wave (128^2 and
// 256^2 cavities) ran 5-10 % slower that way, so they launch normally (the
// kernel's wait then returns at once). After anything but a kernel the
// dependency is the ordinary one.
template <int MINB, typename K, typename... A>
cudaError_t launch_dependent(K kern, dim3 grid, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    const long long blocks = (long long)grid.x * grid.y * grid.z;
    const bool dependent = blocks > (long long)device_sms() * MINB;
    cfg.attrs = dependent ? attr : nullptr;
    cfg.numAttrs = dependent ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename S, int MINB, int TQ, bool BGK>
cudaError_t launch_step4(dim3 grid, cudaStream_t st, const Planes<S> &pl, const Geom &g, const RatesC<float> &r) {
    return launch_dependent<MINB>(k_step4<S, MINB, TQ, BGK>, grid, st, pl, g, r);
}

// The per-warp form: one 128-cell row segment per warp, four per block.
template <typename S, int MINB, int TQ, bool BGK>
cudaError_t launch_step4w(const KParams &p, int src, cudaStream_t st) {
    const int upr = (p.pitch + 127) / 128;
    const long long nunits = (long long)p.ny * upr;
    if (nunits > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((nunits + 3) / 4));
    return launch_dependent<MINB>(k_step4w<S, MINB, TQ, BGK>, grid, st, make_planes<S>(p, src), make_geom(p),
                                  make_rates<float>(p), upr, (int)nunits);
}

// TQ: temperature populations per node (5: D2Q5; 9: the D2Q9 model). BGK:
// single-rate collisions. The D2Q9 model and BGK have the scalar and
// four-cell kernels only.
template <typename S, int TQ, bool BGK>
cudaError_t launch_step_m(const KParams &p, int variant, int src, cudaStream_t st) {
    using C = typename Store<S>::C;
    constexpr bool kBase = TQ == 5 && !BGK;
    if constexpr (Store<S>::kShifted) {
        if (variant == kStepTma) {
            if constexpr (kBase) return launch_tma<S>(p, src, st);
            else return cudaErrorInvalidValue;
        }
        if (variant == kStepVec4) {
            // four cells per thread, 128 threads per block, one row per block row; the
            // config asks ptxas for 4, 5, 6, 7 or 8 resident blocks per SM
            const int threads_x = p.pitch / 4;
            const dim3 grid((threads_x + 127) / 128, p.ny < 65535 ? p.ny : 65535);
            const Planes<S> pl = make_planes<S>(p, src);
            const Geom g = make_geom(p);
            const RatesC<float> r = make_rates<float>(p);
            switch (p.config) {
                case 1: return launch_step4<S, 5, TQ, BGK>(grid, st, pl, g, r);
                case 2: return launch_step4<S, 6, TQ, BGK>(grid, st, pl, g, r);
                case 3: return launch_step4<S, 7, TQ, BGK>(grid, st, pl, g, r);
                case 4: return launch_step4<S, 8, TQ, BGK>(grid, st, pl, g, r);
                default: return launch_step4<S, 4, TQ, BGK>(grid, st, pl, g, r);
            }
        }
        if (variant == kStepVec4w) {
            switch (p.config) {
                case 1: return launch_step4w<S, 5, TQ, BGK>(p, src, st);
                case 2: return launch_step4w<S, 6, TQ, BGK>(p, src, st);
                case 3: return launch_step4w<S, 7, TQ, BGK>(p, src, st);
                case 4: return launch_step4w<S, 8, TQ, BGK>(p, src, st);
                default: return launch_step4w<S, 4, TQ, BGK>(p, src, st);
            }
        }
        if constexpr (sizeof(S) == 2 && kBase) {
            if (variant == kStepVec8) {
                // eight cells per thread (FP16 only)
                const int threads_x = p.pitch / 8;
                const dim3 grid((threads_x + 127) / 128, p.ny < 65535 ? p.ny : 65535);
                const Planes<S> pl = make_planes<S>(p, src);
                const Geom g = make_geom(p);
                const RatesC<float> r = make_rates<float>(p);
                if (p.config == 1) k_step8h<3><<<grid, 128, 0, st>>>(pl, g, r);
                else k_step8h<4><<<grid, 128, 0, st>>>(pl, g, r);
                return cudaGetLastError();
            }
        }
    }
    const dim3 b = step_block();
    const int gy = (p.ny + (int)b.y - 1) / (int)b.y;
    const dim3 grid((p.nx + b.x - 1) / b.x, gy < 65535 ? gy : 65535);
    if (variant != kStepScalar && variant != kStepAuto) return cudaErrorInvalidValue;
    k_step<S, TQ, BGK><<<grid, b, 0, st>>>(make_planes<S>(p, src), make_geom(p), make_rates<C>(p));
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_step_variant(const KParams &p, int variant, int src, cudaStream_t st) {
    if (p.tq == 9)
        return p.bgk ? launch_step_m<S, 9, true>(p, variant, src, st) : launch_step_m<S, 9, false>(p, variant, src, st);
    return p.bgk ? launch_step_m<S, 5, true>(p, variant, src, st) : launch_step_m<S, 5, false>(p, variant, src, st);
}

template <typename S>
cudaError_t launch_init_rows(const KParams &p, int buf, int r0, int r1, const double *T, cudaStream_t st) {
    const dim3 grid((p.pitch + 127) / 128, r1 - r0);
    k_init_rows<S><<<grid, 128, 0, st>>>(make_planes<S>(p, buf), make_geom(p), r0, r1, T, p.T0, p.T_ref, p.varpi,
                                         Store<S>::kShifted ? 1 : 0, p.tq);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_macro_rows(const KParams &p, int buf, int r0, int r1, double *const out[4], cudaStream_t st) {
    using C = typename Store<S>::C;
    const dim3 grid((p.nx + 127) / 128, r1 - r0);
    if (p.tq == 9)
        k_macro_rows<S, 9><<<grid, 128, 0, st>>>(make_planes<S>(p, buf), make_geom(p), make_rates<C>(p), r0, r1,
                                                 p.rho_ref, p.T_ref, out[0], out[1], out[2], out[3]);
    else
        k_macro_rows<S, 5><<<grid, 128, 0, st>>>(make_planes<S>(p, buf), make_geom(p), make_rates<C>(p), r0, r1,
                                                 p.rho_ref, p.T_ref, out[0], out[1], out[2], out[3]);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_export_rows(const KParams &p, int buf, int r0, int r1, double *out, cudaStream_t st) {
    const dim3 grid((p.nx + 127) / 128, r1 - r0);
    k_export_rows<S><<<grid, 128, 0, st>>>(make_planes<S>(p, buf), make_geom(p), r0, r1, p.rho_ref, p.T_ref,
                                           p.varpi, p.tq, out);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_import_rows(const KParams &p, int buf, int r0, int r1, const double *in, int which,
                               cudaStream_t st) {
    const dim3 grid((p.nx + 127) / 128, r1 - r0);
    k_import_rows<S><<<grid, 128, 0, st>>>(make_planes<S>(p, buf), make_geom(p), r0, r1, p.rho_ref, p.T_ref,
                                           p.varpi, p.tq, in, which);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_nusselt(const KParams &p, int buf, int side, double L, double dT, double *partials,
                           cudaStream_t st) {
    if (p.tq == 9)
        k_nusselt<S, 9><<<kRedBlocks, kRedThreads, 0, st>>>(make_planes<S>(p, buf), make_geom(p), side, L, dT,
                                                           p.T_ref, partials);
    else
        k_nusselt<S, 5><<<kRedBlocks, kRedThreads, 0, st>>>(make_planes<S>(p, buf), make_geom(p), side, L, dT,
                                                           p.T_ref, partials);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_residual(const KParams &p, int buf, double *snap, int have_snap, double *partials,
                            cudaStream_t st) {
    using C = typename Store<S>::C;
    if (p.tq == 9)
        k_residual<S, 9><<<kRedBlocks, kRedThreads, 0, st>>>(make_planes<S>(p, buf), make_geom(p), make_rates<C>(p),
                                                            p.T_ref, snap, p.plane, have_snap, partials);
    else
        k_residual<S, 5><<<kRedBlocks, kRedThreads, 0, st>>>(make_planes<S>(p, buf), make_geom(p), make_rates<C>(p),
                                                            p.T_ref, snap, p.plane, have_snap, partials);
    return cudaGetLastError();
}

template <typename S>
Launchers make_launchers() {
    Launchers L;
    L.step = &launch_step<S>;
    L.nee = &launch_nee<S>;
    L.init_rows = &launch_init_rows<S>;
    L.macro_rows = &launch_macro_rows<S>;
    L.export_rows = &launch_export_rows<S>;
    L.import_rows = &launch_import_rows<S>;
    L.nusselt = &launch_nusselt<S>;
    L.residual = &launch_residual<S>;
    return L;
}

}  // namespace nomrt
