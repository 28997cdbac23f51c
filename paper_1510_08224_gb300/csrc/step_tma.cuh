// TMA-staged variant of the fused step (FP32 / FP16-shifted storage).
//
// Work unit: one row segment of W = 512 cells. For each unit one elected
// thread issues 14 bulk copies (cp.async.bulk, one per population plane: the
// row that plane is pulled from, Eq. 9 / Eq. 25, plus a 16-byte halo on each
// side) into a shared-memory stage and arms the stage's mbarrier with the byte
// count. Persistent CTAs walk their units with STAGES stages in flight, so the
// loads of later units overlap the arithmetic of the current one and the
// registers hold only the unit being computed. Stores go straight from
// registers to global memory as 128-bit (FP32) / 64-bit (FP16) vectors.
//
// Every wait on an mbarrier is bounded by a clock budget; on expiry the CTA
// records kStatusTimeout in *status, drains (again bounded) the stages it has
// armed, and returns, so a fault in the copy accounting cannot hang the GPU.
#pragma once

#include "nomrt_kernels.cuh"

namespace nomrt {

constexpr long long kWaitBudgetCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// its later bulk copies (async proxy) into the same shared memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false if the budget ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitBudgetCycles) return false;
    }
    return true;
}

// Row each plane pulls from: planes with e_y = +1 read row y - 1, e_y = -1 read y + 1.
__device__ __forceinline__ int plane_row(int q, int y, int ym, int yp) {
    // f: e_y of directions 0..8 = 0 0 1 0 -1 1 1 -1 -1; g: 0 0 1 0 -1
    switch (q) {
        case 2: case 5: case 6: case 11: return ym;
        case 4: case 7: case 8: case 13: return yp;
        default: return y;
    }
}

struct TmaUnits {
    int y_lo;   // first row with fluid cells possible
    int nrows;  // rows covered
    int nseg;   // segments per row
    int total;  // nrows * nseg
};

// N consecutive storage elements <-> N compute values.
template <typename S, int N>
struct VecN;

template <typename S>
struct VecN<S, 4> {
    static __device__ __forceinline__ void ld_shared(const S *p, float a[4]) { Vec4<S>::ld_shared(p, a); }
    static __device__ __forceinline__ void st(S *p, const float a[4]) { Vec4<S>::st(p, a); }
};

template <>
struct VecN<float, 2> {
    static __device__ __forceinline__ void ld_shared(const float *p, float a[2]) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        a[0] = v.x; a[1] = v.y;
    }
    static __device__ __forceinline__ void st(float *p, const float a[2]) {
        *reinterpret_cast<float2 *>(p) = make_float2(a[0], a[1]);
    }
};

template <>
struct VecN<__half, 2> {
    static __device__ __forceinline__ void ld_shared(const __half *p, float a[2]) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(p));
        a[0] = f.x; a[1] = f.y;
    }
    static __device__ __forceinline__ void st(__half *p, const float a[2]) {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a[0], a[1]);
    }
};

template <typename S>
struct VecN<S, 1> {
    static __device__ __forceinline__ void ld_shared(const S *p, float a[1]) { a[0] = (float)p[0]; }
    static __device__ __forceinline__ void st(S *p, const float a[1]) { Store<S>::st(p, a[0]); }
};

// Link-map bytes of N consecutive cells (N-byte aligned), packed little-endian.
template <int N>
__device__ __forceinline__ uint32_t ld_mask(const uint8_t *p) {
    if (N == 4) return __ldg(reinterpret_cast<const uint32_t *>(p));
    if (N == 2) return (uint32_t)__ldg(reinterpret_cast<const uint16_t *>(p));
    return (uint32_t)__ldg(p);
}

template <int N>
__host__ __device__ constexpr uint32_t all_solid() {
    return N == 4 ? 0xFFFFFFFFu : (N == 2 ? 0xFFFFu : 0xFFu);
}

// Issue the 14 copies of unit u into a stage (one elected thread).
template <typename S, int W>
__device__ __forceinline__ void tma_issue(const Planes<S> &pl, const Geom &g, const TmaUnits &U, int u, S *stage,
                                          uint64_t *bar) {
    constexpr int HALO = 16 / (int)sizeof(S);
    constexpr int ROW = W + 2 * HALO;
    const int y = U.y_lo + u / U.nseg;
    const int xs = (u % U.nseg) * W;
    int ym = y - 1, yp = y + 1;
    if (g.py) {
        ym = (ym < 0) ? ym + g.ny : ym;
        yp = (yp >= g.ny) ? yp - g.ny : yp;
    }
    const int lo = xs - HALO < 0 ? 0 : xs - HALO;
    const int hi = xs + W + HALO > g.pitch ? g.pitch : xs + W + HALO;
    const uint32_t bytes = (uint32_t)((hi - lo) * (int)sizeof(S));
    // the barrier expects the bytes of the copies that are issued (all of them, except where the
    // bounds-checking build refuses a source range)
    uint32_t armed_bytes = bytes * kQ;
    if constexpr (kBoundsBuild) {
        armed_bytes = 0;
        for (int q = 0; q < kQ; ++q)
            if (NOMRT_BULK_OK(g, pl.src[q] + (size_t)plane_row(q, y, ym, yp) * g.pitch + lo, bytes, 40))
                armed_bytes += bytes;
    }
    mbar_arrive_expect_tx(bar, armed_bytes);
#pragma unroll 1
    for (int q = 0; q < kQ; ++q) {
        const S *src = pl.src[q] + (size_t)plane_row(q, y, ym, yp) * g.pitch + lo;
        S *dst = stage + q * ROW + (lo - (xs - HALO));
        if (!kBoundsBuild || NOMRT_BULK_OK(g, src, bytes, 40)) bulk_g2s(dst, src, bytes, bar);
    }
}

// N values of one plane for cells x0..x0+N-1 from the staged row `sm`
// (sm[HALO + j] holds cell xs + j), with the pull rules of ld_plane: DX = +1
// pulls from x - 1, DX = -1 from x + 1; the periodic seam reads global memory.
template <typename S, int DX, int N>
__device__ __forceinline__ void sm_plane(const S *sm, const S *grow, const Geom &g, int j0, int x0, int lane,
                                         float out[N]) {
    constexpr int HALO = 16 / (int)sizeof(S);
    if (N == 1) {
        out[0] = (float)sm[HALO + j0 - DX];
    } else {
        float a[N];
        VecN<S, N>::ld_shared(sm + HALO + j0, a);
        if (DX == 0) {
#pragma unroll
            for (int k = 0; k < N; ++k) out[k] = a[k];
        } else if (DX == 1) {
            float left = __shfl_up_sync(kFull, a[N - 1], 1);
            if (lane == 0) left = (float)sm[HALO + j0 - 1];
            out[0] = left;
#pragma unroll
            for (int k = 1; k < N; ++k) out[k] = a[k - 1];
        } else {
            float right = __shfl_down_sync(kFull, a[0], 1);
            if (lane == 31) right = (float)sm[HALO + j0 + N];
#pragma unroll
            for (int k = 0; k < N - 1; ++k) out[k] = a[k + 1];
            out[N - 1] = right;
        }
    }
    if (DX == 1 && g.px && x0 == 0) out[0] = ld_at<S>(g, grow + g.nx - 1, 41);  // periodic seam
    if (DX == -1 && g.px) {
        const int k = g.nx - 1 - x0;
        if (k >= 0 && k < N) {
            const float v = ld_at<S>(g, grow, 42);  // periodic seam: x = nx - 1 pulls from x = 0
#pragma unroll
            for (int j = 0; j < N; ++j) out[j] = (j == k) ? v : out[j];  // constant indices only
        }
    }
}

// Wall links, collision and solid zeroing of an N-cell group: pairs of cells
// collide as float2, a single cell as float.
template <typename S, int N>
__device__ __forceinline__ void cells_N(const Planes<S> &pl, const Geom &g, const RatesC<float> &r, uint32_t mN,
                                        int x0, int r0, int rm, int rp, float f[9][N], float t[5][N]) {
    if (mN != 0u) {
        wall_links<S, 0, N>(pl, g, mN, x0, r0, rm, rp, f, t);
        if constexpr (N >= 2) wall_links<S, 1, N>(pl, g, mN, x0, r0, rm, rp, f, t);
        if constexpr (N >= 4) {
            wall_links<S, 2, N>(pl, g, mN, x0, r0, rm, rp, f, t);
            wall_links<S, 3, N>(pl, g, mN, x0, r0, rm, rp, f, t);
        }
    }
    if constexpr (N == 1) {
        float fk[9], tk[5];
#pragma unroll
        for (int i = 0; i < 9; ++i) fk[i] = f[i][0];
#pragma unroll
        for (int i = 0; i < 5; ++i) tk[i] = t[i][0];
        collide_x<float>(r, fk, tk);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i][0] = fk[i];
#pragma unroll
        for (int i = 0; i < 5; ++i) t[i][0] = tk[i];
    } else {
        collide_pair<0, N>(r, f, t);
        if constexpr (N >= 4) collide_pair<2, N>(r, f, t);
    }
    if (mN != 0u) {
        zero_solid<0, N>(mN, f, t);
        if constexpr (N >= 2) zero_solid<1, N>(mN, f, t);
        if constexpr (N >= 4) {
            zero_solid<2, N>(mN, f, t);
            zero_solid<3, N>(mN, f, t);
        }
    }
}

// Shape of a TMA step kernel: N cells per thread, T threads per CTA (a unit of
// W = N * T cells), STAGES pipeline stages, MINB CTAs per SM asked of ptxas.
template <typename S, int N, int T, int STAGES, int MINB>
__global__ void __launch_bounds__(T, MINB) k_step_tma(const Planes<S> pl, const Geom g, const RatesC<float> r,
                                                      const TmaUnits U, int *status) {
    constexpr int W = N * T;
    constexpr int HALO = 16 / (int)sizeof(S);
    constexpr int ROW = W + 2 * HALO;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S *stages = reinterpret_cast<S *>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + (size_t)STAGES * kQ * ROW * sizeof(S));
    __shared__ int abort_flag;

    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    // prologue: arm the first STAGES units of this CTA
    int armed = 0;  // units issued (thread 0's view)
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            const int u = blockIdx.x + s * gridDim.x;
            if (u >= U.total) break;
            tma_issue<S, W>(pl, g, U, u, stages + (size_t)s * kQ * ROW, &bars[s]);
            ++armed;
        }
    }
    int i = 0;
    for (int u = blockIdx.x; u < U.total; u += gridDim.x, ++i) {
        const int s = i % STAGES;
        const uint32_t parity = (uint32_t)((i / STAGES) & 1);
        if (!mbar_wait_bounded(&bars[s], parity)) atomicExch(&abort_flag, 1);
        __syncthreads();
        if (abort_flag) break;
        const S *st = stages + (size_t)s * kQ * ROW;
        const int y = U.y_lo + u / U.nseg;
        const int xs = (u % U.nseg) * W;
        const int j0 = tid * N;
        const int x0 = xs + j0;
        const int r0 = y * g.pitch;
        int ym = y - 1, yp = y + 1;
        if (g.py) {
            ym = (ym < 0) ? ym + g.ny : ym;
            yp = (yp >= g.ny) ? yp - g.ny : yp;
        }
        const int rm = ym * g.pitch, rp = yp * g.pitch;
        const bool inrow = x0 < g.pitch;
        uint32_t mN = all_solid<N>();
        if (inrow && NOMRT_OK(g, g.mask + r0 + x0, N, 43)) mN = ld_mask<N>(g.mask + r0 + x0);
        const bool any = mN != all_solid<N>();
        if (__any_sync(kFull, any)) {
            float f[9][N], t[5][N];
            sm_plane<S, 0, N>(st + 0 * ROW, pl.src[0] + r0, g, j0, x0, lane, f[0]);
            sm_plane<S, 1, N>(st + 1 * ROW, pl.src[1] + r0, g, j0, x0, lane, f[1]);
            sm_plane<S, 0, N>(st + 2 * ROW, pl.src[2] + rm, g, j0, x0, lane, f[2]);
            sm_plane<S, -1, N>(st + 3 * ROW, pl.src[3] + r0, g, j0, x0, lane, f[3]);
            sm_plane<S, 0, N>(st + 4 * ROW, pl.src[4] + rp, g, j0, x0, lane, f[4]);
            sm_plane<S, 1, N>(st + 5 * ROW, pl.src[5] + rm, g, j0, x0, lane, f[5]);
            sm_plane<S, -1, N>(st + 6 * ROW, pl.src[6] + rm, g, j0, x0, lane, f[6]);
            sm_plane<S, -1, N>(st + 7 * ROW, pl.src[7] + rp, g, j0, x0, lane, f[7]);
            sm_plane<S, 1, N>(st + 8 * ROW, pl.src[8] + rp, g, j0, x0, lane, f[8]);
            sm_plane<S, 0, N>(st + 9 * ROW, pl.src[9] + r0, g, j0, x0, lane, t[0]);
            sm_plane<S, 1, N>(st + 10 * ROW, pl.src[10] + r0, g, j0, x0, lane, t[1]);
            sm_plane<S, 0, N>(st + 11 * ROW, pl.src[11] + rm, g, j0, x0, lane, t[2]);
            sm_plane<S, -1, N>(st + 12 * ROW, pl.src[12] + r0, g, j0, x0, lane, t[3]);
            sm_plane<S, 0, N>(st + 13 * ROW, pl.src[13] + rp, g, j0, x0, lane, t[4]);
            if (any) {
                cells_N<S, N>(pl, g, r, mN, x0, r0, rm, rp, f, t);
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    if (NOMRT_OK(g, pl.dst[q] + r0 + x0, N * sizeof(S), 44)) VecN<S, N>::st(pl.dst[q] + r0 + x0, f[q]);
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    if (NOMRT_OK(g, pl.dst[9 + q] + r0 + x0, N * sizeof(S), 44))
                        VecN<S, N>::st(pl.dst[9 + q] + r0 + x0, t[q]);
            }
        }
        // every thread is done reading stage s: refill it with this CTA's unit STAGES ahead
        __syncthreads();
        if (tid == 0) {
            const int un = u + STAGES * gridDim.x;
            if (un < U.total) {
                fence_proxy_async_smem();
                tma_issue<S, W>(pl, g, U, un, stages + (size_t)s * kQ * ROW, &bars[s]);
                ++armed;
            }
        }
    }
    if (abort_flag && tid == 0) {
        atomicExch(status, kStatusTimeout);
        // drain: wait (bounded) for every armed stage not yet consumed before the CTA's
        // shared memory is released
        for (int k = i; k < armed; ++k) mbar_wait_bounded(&bars[k % STAGES], (uint32_t)((k / STAGES) & 1));
    }
}

}  // namespace nomrt
