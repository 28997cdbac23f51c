// Device code of the fused non-orthogonal MRT stream-and-collide update
// (Liu, He, Li & Li, arXiv:1510.08224, Sec. 2), templated on the population
// storage type. Included once by each of kernels_f64.cu, kernels_f32.cu and
// kernels_f16.cu, which instantiate it and fill a Launchers table.
//
// Data layout in HBM (structure of arrays, ping-pong):
//   pop[b] = kQ planes of ny rows x pitch elements; planes 0..8 hold f_bar_i,
//   planes 9..13 hold g_i, in the direction order of Eq. 5. pitch is nx rounded
//   up to a 128-byte multiple. A node is read from the source buffer by the pull
//   form of the streaming steps (Eqs. 9, 25): f_bar_i(x) <- f_bar*_i(x - e_i),
//   collided in registers, and written back at x in the other buffer.
//
// Arithmetic: the 9x9 map of Eq. 13 and its inverse (Eq. A1) are applied as
// add/sub chains on shared pair sums; the 1/2 and 1/4 of Eq. A1 are exact
// scalings. No tensor cores: each node is a separate 9-vector.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "nomrt_internal.h"

namespace nomrt {

// ------------------------------------------------------------ storage traits

template <typename S>
struct Store;

template <>
struct Store<double> {
    using C = double;
    static constexpr bool kShifted = false;
    static __device__ __forceinline__ C ld(const double *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(double *p, C v) { *p = v; }
};

template <>
struct Store<float> {
    using C = float;
    static constexpr bool kShifted = true;
    static __device__ __forceinline__ C ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float *p, C v) { *p = v; }
};

template <>
struct Store<__half> {
    using C = float;
    static constexpr bool kShifted = true;
    static __device__ __forceinline__ C ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st(__half *p, C v) { *p = __float2half_rn(v); }
};

// Population loads of a step. NC = true: the read-only data path (the
// source buffer is never written by the same launch). NC = false: L2-coherent
// loads (ld.global.cg) for kernels that run several steps in one launch and
// so read data the same launch wrote.
template <typename S, bool NC>
struct Ld;

template <bool NC>
struct Ld<float, NC> {
    static __device__ __forceinline__ float one(const float *p) { return NC ? __ldg(p) : __ldcg(p); }
    static __device__ __forceinline__ void four(const float *p, float a[4]) {
        const float4 v = NC ? __ldg(reinterpret_cast<const float4 *>(p)) : __ldcg(reinterpret_cast<const float4 *>(p));
        a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
    }
};

template <bool NC>
struct Ld<__half, NC> {
    static __device__ __forceinline__ float one(const __half *p) {
        return __half2float(NC ? __ldg(p) : __ldcg(p));
    }
    static __device__ __forceinline__ void four(const __half *p, float a[4]) {
        const uint2 v = NC ? __ldg(reinterpret_cast<const uint2 *>(p)) : __ldcg(reinterpret_cast<const uint2 *>(p));
        __half2 h0, h1;
        memcpy(&h0, &v.x, 4);
        memcpy(&h1, &v.y, 4);
        const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
        a[0] = f0.x; a[1] = f0.y; a[2] = f1.x; a[3] = f1.y;
    }
};

// Rates and constants in the compute type, precomputed once per launch on the
// host side of the launcher.
template <typename C>
struct RatesC {
    C om_e, om_nu, om_q, om_eps;  // 1 - s_k
    C s_e, s_nu, s_q, s_eps;      // s_k
    C h_e, h_nu, h_eps;           // 1 - s_k / 2
    C om_a, z_a, om_ze, zv_e, om_zn;  // thermal: 1 - zeta_alpha, zeta_alpha, 1 - zeta_e, zeta_e varpi, 1 - zeta_nu
    C ax, Fy0, g_beta;            // F = (ax, Fy0 + g_beta (T - T_ref))
    C T_ref;
    C hx;                         // ax / 2
    C h2e, h2nu, h23eps;          // 2 (1 - s_e/2), 2 (1 - s_nu/2), (2/3)(1 - s_eps/2)
    C varpi;                      // Eq. 28
    // D2Q9 temperature model (Eqs. 31-33): zeta_e, zeta_nu, zeta_q, zeta_eps and theta
    C z_e, z_nu, om_zq, z_q, om_zeps, z_eps, theta;
};

template <typename C>
inline RatesC<C> make_rates(const KParams &p) {
    RatesC<C> r;
    r.s_e = (C)p.s_e;
    r.s_nu = (C)p.s_nu;
    r.s_q = (C)p.s_q;
    r.s_eps = (C)p.s_eps;
    r.om_e = (C)(1.0 - p.s_e);
    r.om_nu = (C)(1.0 - p.s_nu);
    r.om_q = (C)(1.0 - p.s_q);
    r.om_eps = (C)(1.0 - p.s_eps);
    r.h_e = (C)(1.0 - 0.5 * p.s_e);
    r.h_nu = (C)(1.0 - 0.5 * p.s_nu);
    r.h_eps = (C)(1.0 - 0.5 * p.s_eps);
    r.om_a = (C)(1.0 - p.z_a);
    r.z_a = (C)p.z_a;
    r.om_ze = (C)(1.0 - p.z_e);
    r.zv_e = (C)(p.z_e * p.varpi);
    r.om_zn = (C)(1.0 - p.z_nu);
    r.ax = (C)p.ax;
    r.Fy0 = (C)(p.ay + p.g_beta * (p.T_ref - p.T0));
    r.g_beta = (C)p.g_beta;
    r.T_ref = (C)p.T_ref;
    r.hx = (C)(0.5 * p.ax);
    r.h2e = (C)(2.0 * (1.0 - 0.5 * p.s_e));
    r.h2nu = (C)(2.0 * (1.0 - 0.5 * p.s_nu));
    r.h23eps = (C)(2.0 / 3.0 * (1.0 - 0.5 * p.s_eps));
    r.varpi = (C)p.varpi;
    r.z_e = (C)p.z_e;
    r.z_nu = (C)p.z_nu;
    r.om_zq = (C)(1.0 - p.z_q);
    r.z_q = (C)p.z_q;
    r.om_zeps = (C)(1.0 - p.z_eps);
    r.z_eps = (C)p.z_eps;
    r.theta = (C)p.theta;
    return r;
}

// Kernel arguments: typed plane pointers of both buffers.
template <typename S>
struct Planes {
    const S *src[kQmax];
    S *dst[kQmax];
    __device__ __forceinline__ const S *src_at(int q) const { return src[q]; }
    __device__ __forceinline__ S *dst_at(int q) const { return dst[q]; }
};

template <typename S>
inline Planes<S> make_planes(const KParams &p, int src) {
    Planes<S> pl;
    S *a = static_cast<S *>(p.pop[src]);
    S *b = static_cast<S *>(p.pop[1 - src]);
    for (int q = 0; q < kQmax; ++q) {
        pl.src[q] = a + (size_t)q * p.plane;
        pl.dst[q] = b + (size_t)q * p.plane;
    }
    return pl;
}

struct Geom {
    int nx, ny, pitch, px, py;
    const uint8_t *mask;
    const uint8_t *flags;
    const WallDev *walls;
    const uint8_t *nee_dir;  // per cell: 0, or the direction of a boundary node's nearest fluid node
    const char *lo, *hi;     // the lattice's device block (checked by the bounds-checking build)
    int *oob;                // first failing check's site id (bounds-checking build)
};

inline Geom make_geom(const KParams &p) {
    return Geom{p.nx, p.ny, p.pitch, p.px, p.py, p.mask, p.flags, p.walls, p.nee_dir, p.blk_lo, p.blk_hi, p.oob};
}

// ------------------------------------------------------------- index checks

// The bounds-checking build (-DLBM_BOUNDS) tests every population, map and
// wall-table access of the step kernels before making it: the bytes
// [p, p + bytes) must lie in the lattice's device block and a 2-, 4-, 8- or
// 16-byte access must be aligned to its size. An access that fails is
// skipped (a load reads 0) and the first failing site id is recorded in the
// lattice's bounds word, which the synchronising calls report; nothing traps.
// The sites: 1-9 pull / scalar kernel, 10-19 four-cell rows, 20-29 wall
// links and node pass, 30-39 eight-cell kernel, 40-49 TMA kernel, 50-59
// prefetches. Without LBM_BOUNDS every check is the constant true.
#ifdef LBM_BOUNDS
static __device__ __noinline__ void oob_note(int *w, int site) { atomicCAS(w, 0, site); }

__device__ __forceinline__ bool in_block(const Geom &g, const void *p, int bytes, int site) {
    const char *c = static_cast<const char *>(p);
    const bool pow2 = (bytes & (bytes - 1)) == 0;
    const bool ok = c >= g.lo && c + bytes <= g.hi &&
                    (!pow2 || bytes > 16 || (reinterpret_cast<uintptr_t>(c) & (uintptr_t)(bytes - 1)) == 0);
    if (!ok) oob_note(g.oob, site);
    return ok;
}
#define NOMRT_OK(g, p, bytes, site) ::nomrt::in_block((g), (p), (int)(bytes), (site))
#else
#define NOMRT_OK(g, p, bytes, site) true
#endif

// A bulk copy or prefetch of `bytes` at p: in the block, 16-byte aligned, a
// multiple of 16 bytes.
#define NOMRT_BULK_OK(g, p, bytes, site) \
    (NOMRT_OK(g, p, bytes, site) && ((reinterpret_cast<uintptr_t>(p) & 15u) == 0 && ((bytes) & 15u) == 0))

// A cell whose populations are kept: fluid, or a boundary node of an NEE wall.
__device__ __forceinline__ bool kept_cell(const Geom &g, int off) {
    return g.mask[off] != kSolid || g.nee_dir[off] != 0;
}

// --------------------------------------------------------------- pull step

// One population value at p (0 where the bounds-checking build refuses p).
template <typename S>
__device__ __forceinline__ typename Store<S>::C ld_at(const Geom &g, const S *p, int site) {
    if (!NOMRT_OK(g, p, sizeof(S), site)) return typename Store<S>::C(0);
    return Store<S>::ld(p);
}

// The wall-table entry of the wall that cell `off` belongs to (nullptr where
// the bounds-checking build refuses the flag or the entry).
__device__ __forceinline__ const WallDev *wall_of(const Geom &g, int off, int site) {
    if (!NOMRT_OK(g, g.flags + off, 1, site)) return nullptr;
    const WallDev *w = g.walls + g.flags[off];
    if (!NOMRT_OK(g, w, sizeof(WallDev), site)) return nullptr;
    return w;
}

// Post-streaming populations at fluid cell (x, y): Eq. 9 and Eq. 25 in pull
// form, then the halfway wall rules on the links flagged in `m`.
template <typename S, int TQ = 5>
__device__ __forceinline__ void pull(const S *const *src, const Geom &g, int x, int y, unsigned m,
                                     typename Store<S>::C f[9], typename Store<S>::C t[TQ]) {
    using St = Store<S>;
    int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1;
    if (g.px) {
        xm = (xm < 0) ? xm + g.nx : xm;
        xp = (xp >= g.nx) ? xp - g.nx : xp;
    }
    if (g.py) {
        ym = (ym < 0) ? ym + g.ny : ym;
        yp = (yp >= g.ny) ? yp - g.ny : yp;
    }
    const int r0 = y * g.pitch, rm = ym * g.pitch, rp = yp * g.pitch;
    // direction i pulls from x - e_i (Eq. 5 numbering)
    f[0] = ld_at<S>(g, src[0] + r0 + x, 1);
    f[1] = ld_at<S>(g, src[1] + r0 + xm, 1);
    f[2] = ld_at<S>(g, src[2] + rm + x, 1);
    f[3] = ld_at<S>(g, src[3] + r0 + xp, 1);
    f[4] = ld_at<S>(g, src[4] + rp + x, 1);
    f[5] = ld_at<S>(g, src[5] + rm + xm, 1);
    f[6] = ld_at<S>(g, src[6] + rm + xp, 1);
    f[7] = ld_at<S>(g, src[7] + rp + xp, 1);
    f[8] = ld_at<S>(g, src[8] + rp + xm, 1);
    t[0] = ld_at<S>(g, src[9] + r0 + x, 2);
    t[1] = ld_at<S>(g, src[10] + r0 + xm, 2);
    t[2] = ld_at<S>(g, src[11] + rm + x, 2);
    t[3] = ld_at<S>(g, src[12] + r0 + xp, 2);
    t[4] = ld_at<S>(g, src[13] + rp + x, 2);
    if constexpr (TQ == 9) {
        t[5] = ld_at<S>(g, src[14] + rm + xm, 2);
        t[6] = ld_at<S>(g, src[15] + rm + xp, 2);
        t[7] = ld_at<S>(g, src[16] + rp + xp, 2);
        t[8] = ld_at<S>(g, src[17] + rp + xm, 2);
    }
    if (m) {
        using C = typename St::C;
        const int sidx[9] = {r0 + x, r0 + xm, rm + x, r0 + xp, rp + x, rm + xm, rm + xp, rp + xp, rp + xm};
        const int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (m & (1u << (i - 1))) {
                const WallDev *w = wall_of(g, sidx[i], 3);
                if (kBoundsBuild && !w) continue;
                f[i] = ld_at<S>(g, src[opp[i]] + r0 + x, 4) + (C)__ldg(&w->cf[i]);
                if (i < TQ)
                    t[i] = (C)__ldg(&w->tsgn) * ld_at<S>(g, src[9 + opp[i]] + r0 + x, 5) +
                           (C)__ldg(TQ == 9 ? &w->tb9[i] : &w->tb);
            }
        }
    }
}

// ------------------------------------------------------------- collisions

// Macroscopic values from post-streaming populations (Eqs. 4, 18, 19, 27) in
// the storage's frame: returns d_rho = rho - rho_ref, u, dT = T - T_ref, F.
template <typename C>
struct Macro {
    C drho, ux, uy, dT, Fx, Fy;
};

template <typename C, int TQ = 5>
__device__ __forceinline__ Macro<C> macro_of(const RatesC<C> &r, const C f[9], const C t[TQ]) {
    Macro<C> M;
    if constexpr (TQ == 9) M.dT = (((t[0] + t[1]) + (t[2] + t[3])) + (t[4] + t[5])) + ((t[6] + t[7]) + t[8]);
    else M.dT = ((t[0] + t[1]) + (t[2] + t[3])) + t[4];
    M.Fx = r.ax;
    M.Fy = r.Fy0 + r.g_beta * M.dT;
    M.drho = (((f[0] + f[1]) + (f[2] + f[3])) + (f[4] + f[5])) + ((f[6] + f[7]) + f[8]);
    const C jx = (f[1] - f[3]) + ((f[5] - f[7]) - (f[6] - f[8]));
    const C jy = (f[2] - f[4]) + ((f[5] - f[7]) + (f[6] - f[8]));
    M.ux = jx + C(0.5) * M.Fx;
    M.uy = jy + C(0.5) * M.Fy;
    return M;
}

// Non-equilibrium extrapolation at boundary node (x, y) of wall w whose nearest
// fluid node is x + e_d: the fluid node's post-streaming populations plus the
// difference of the equilibria at the wall state and at the fluid node's
// state (Eq. 22 under the incompressible reading; Eq. 30), which is
//   f_b = f_eq(rho_f, u_w) + [f(x_f) - f_eq(rho_f, u_f)]
//   g_b = g_eq(T_b, u_w)   + [g(x_f) - g_eq(T_f, u_f)]
// in the storage frame (the shift cancels in the differences).
template <typename S, int TQ = 5>
__device__ __forceinline__ void nee_rebuild(const S *const *src, const Geom &g,
                                            const RatesC<typename Store<S>::C> &r, int x, int y, int d,
                                            const WallDev *w, typename Store<S>::C f[9],
                                            typename Store<S>::C t[TQ]) {
    using C = typename Store<S>::C;
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const C w9[9] = {C(4.0 / 9), C(1.0 / 9), C(1.0 / 9), C(1.0 / 9), C(1.0 / 9),
                     C(1.0 / 36), C(1.0 / 36), C(1.0 / 36), C(1.0 / 36)};
    int xf = x + ex[d], yf = y + ey[d];
    if (g.px) xf = (xf < 0) ? xf + g.nx : (xf >= g.nx ? xf - g.nx : xf);
    if (g.py) yf = (yf < 0) ? yf + g.ny : (yf >= g.ny ? yf - g.ny : yf);
    const unsigned mf = NOMRT_OK(g, g.mask + yf * g.pitch + xf, 1, 20) ? g.mask[yf * g.pitch + xf] : 0u;
    pull<S, TQ>(src, g, xf, yf, mf, f, t);
    const Macro<C> M = macro_of<C, TQ>(r, f, t);
    const C uwx = (C)w->uwx, uwy = (C)w->uwy;
    const C Tf = r.T_ref + M.dT;
    const C Tb = w->adiabatic != 0.0 ? Tf : (C)w->Tw;
    const C uf2 = M.ux * M.ux + M.uy * M.uy, uw2 = uwx * uwx + uwy * uwy;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const C euw = ex[i] * uwx + ey[i] * uwy, euf = ex[i] * M.ux + ey[i] * M.uy;
        f[i] += w9[i] * ((C(3) * euw + C(4.5) * euw * euw - C(1.5) * uw2) -
                         (C(3) * euf + C(4.5) * euf * euf - C(1.5) * uf2));
    }
    if constexpr (TQ == 9) {
        // Eq. 31 at (T_b, u_w) and (T_f, u_f)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const C euw = ex[i] * uwx + ey[i] * uwy, euf = ex[i] * M.ux + ey[i] * M.uy;
            t[i] += w9[i] * (Tb * (C(1) + C(3) * euw + r.theta * (C(4.5) * euw * euw - C(1.5) * uw2)) -
                             Tf * (C(1) + C(3) * euf + r.theta * (C(4.5) * euf * euf - C(1.5) * uf2)));
        }
    } else {
        t[0] += (C(1) - r.varpi) * (Tb - Tf);
#pragma unroll
        for (int i = 1; i < 5; ++i) {
            const C euw = ex[i] * uwx + ey[i] * uwy, euf = ex[i] * M.ux + ey[i] * M.uy;
            t[i] += C(0.25) * r.varpi * (Tb - Tf) + C(0.5) * (euw * Tb - euf * Tf);
        }
    }
}

// Flow collision (Eq. 8 with Eqs. 16, 17, 20 under the incompressible reading,
// rho0 = 1) and temperature collision (Eq. 24 with Eqs. 28, 29), in place.
// D2Q9 temperature model (Eqs. 31-33, reading: the transformation is M of
// Eq. 13): n = M g on pair sums, n* = n - Q (n - n_eq) with n_eq = M g_eq of
// Eq. 31 in the storage frame, g = M^-1 n*. n0 = T - T_ref is given.
template <typename C>
__device__ __forceinline__ void thermal_q9(const RatesC<C> &r, C t[9], C n0, C ux, C uy, C uu) {
    const C b13 = t[1] + t[3], e13 = t[1] - t[3];
    const C b24 = t[2] + t[4], e24 = t[2] - t[4];
    const C b57 = t[5] + t[7], e57 = t[5] - t[7];
    const C b68 = t[6] + t[8], e68 = t[6] - t[8];
    const C Dt = b57 + b68;
    const C n6 = e57 + e68, n7 = e57 - e68;
    const C n1 = e13 + n7, n2 = e24 + n6;
    const C n3 = (b13 + b24) + (Dt + Dt);
    const C n4 = b13 - b24, n5 = b57 - b68, n8 = Dt;
    const C T = r.T_ref + n0;
    const C q1 = r.om_a * n1 + r.z_a * (T * ux);
    const C q2 = r.om_a * n2 + r.z_a * (T * uy);
    const C q3 = r.om_ze * n3 + r.z_e * (C(2.0 / 3.0) * n0 + r.theta * (T * uu));
    const C q4 = r.om_zn * n4 + r.z_nu * (r.theta * (T * (ux * ux - uy * uy)));
    const C q5 = r.om_zn * n5 + r.z_nu * (r.theta * (T * (ux * uy)));
    const C q6 = r.om_zq * n6 + r.z_q * (C(1.0 / 3.0) * (T * uy));
    const C q7 = r.om_zq * n7 + r.z_q * (C(1.0 / 3.0) * (T * ux));
    const C q8 = r.om_zeps * n8 + r.z_eps * (C(1.0 / 9.0) * n0 + C(1.0 / 3.0) * (r.theta * (T * uu)));
    const C A = C(0.25) * q3 - C(0.5) * q8;
    const C B = C(0.25) * q4;
    const C h1 = C(0.5) * (q1 - q7);
    const C h2 = C(0.5) * (q2 - q6);
    const C P = C(0.25) * (q8 + q5);
    const C Q = C(0.25) * (q6 + q7);
    const C R = C(0.25) * (q8 - q5);
    const C Sx = C(0.25) * (q6 - q7);
    t[0] = (n0 - q3) + q8;
    t[1] = (A + B) + h1;
    t[3] = (A + B) - h1;
    t[2] = (A - B) + h2;
    t[4] = (A - B) - h2;
    t[5] = P + Q;
    t[7] = P - Q;
    t[6] = R + Sx;
    t[8] = R - Sx;
}

template <typename C, int TQ = 5>
__device__ __forceinline__ void collide(const RatesC<C> &r, C f[9], C t[TQ]) {
    // temperature first: the buoyancy of Eq. 4 needs it
    C n0;
    if constexpr (TQ == 9) n0 = (((t[0] + t[1]) + (t[2] + t[3])) + (t[4] + t[5])) + ((t[6] + t[7]) + t[8]);
    else n0 = ((t[0] + t[1]) + (t[2] + t[3])) + t[4];  // T - T_ref
    const C Fx = r.ax;
    const C Fy = r.Fy0 + r.g_beta * n0;  // Eq. 4

    // ---- D2Q9 forward map m = M f (Eq. 13) on pair sums
    const C a13 = f[1] + f[3], d13 = f[1] - f[3];
    const C a24 = f[2] + f[4], d24 = f[2] - f[4];
    const C a57 = f[5] + f[7], d57 = f[5] - f[7];
    const C a68 = f[6] + f[8], d68 = f[6] - f[8];
    const C D = a57 + a68;
    const C m0 = (f[0] + (a13 + a24)) + D;  // rho - rho_ref
    const C m6 = d57 + d68;
    const C m7 = d57 - d68;
    const C jx = d13 + m7;
    const C jy = d24 + m6;
    const C m3 = (a13 + a24) + (D + D);
    const C m4 = a13 - a24;
    const C m5 = a57 - a68;
    const C m8 = D;

    // Eq. 19 with rho0 = 1
    const C ux = jx + C(0.5) * Fx;
    const C uy = jy + C(0.5) * Fy;
    const C uu = ux * ux + uy * uy;
    const C uF = ux * Fx + uy * Fy;

    // ---- Eq. 8: m* = (1 - s) m + s m_eq + (1 - s/2) S~
    const C p1 = jx + Fx;  // any s1: conserved moment plus the force impulse
    const C p2 = jy + Fy;
    const C p3 = r.om_e * m3 + r.s_e * (C(2.0 / 3.0) * m0 + uu) + r.h_e * (C(2) * uF);
    const C p4 = r.om_nu * m4 + r.s_nu * (ux * ux - uy * uy) + r.h_nu * (C(2) * (ux * Fx - uy * Fy));
    const C p5 = r.om_nu * m5 + r.s_nu * (ux * uy) + r.h_nu * (ux * Fy + uy * Fx);
    // s_q m_eq + (1 - s_q/2) S~ for q_xxy, q_xyy reduces to (s_q j + F) / 3
    const C p6 = r.om_q * m6 + C(1.0 / 3.0) * (r.s_q * jy + Fy);
    const C p7 = r.om_q * m7 + C(1.0 / 3.0) * (r.s_q * jx + Fx);
    const C p8 = r.om_eps * m8 + r.s_eps * (C(1.0 / 9.0) * m0 + C(1.0 / 3.0) * uu) + r.h_eps * (C(2.0 / 3.0) * uF);

    // ---- back map f = M^-1 m* (Eq. A1)
    const C A = C(0.25) * p3 - C(0.5) * p8;
    const C B = C(0.25) * p4;
    const C h1 = C(0.5) * (p1 - p7);
    const C h2 = C(0.5) * (p2 - p6);
    const C P = C(0.25) * (p8 + p5);
    const C Q = C(0.25) * (p6 + p7);
    const C R = C(0.25) * (p8 - p5);
    const C Sx = C(0.25) * (p6 - p7);
    f[0] = (m0 - p3) + p8;
    f[1] = (A + B) + h1;
    f[3] = (A + B) - h1;
    f[2] = (A - B) + h2;
    f[4] = (A - B) - h2;
    f[5] = P + Q;
    f[7] = P - Q;
    f[6] = R + Sx;
    f[8] = R - Sx;

    if constexpr (TQ == 9) {
        thermal_q9<C>(r, t, n0, ux, uy, uu);
        return;
    } else {
    // ---- D2Q5: n = N g (Eq. 26), relaxation (Eq. 24) with n_eq = (T, ux T, uy T, varpi T, 0),
    // g = N^-1 n* (Eq. A2)
    const C n1 = t[1] - t[3];
    const C n2 = t[2] - t[4];
    const C n3 = (t[1] + t[3]) + (t[2] + t[4]);
    const C n4 = (t[1] + t[3]) - (t[2] + t[4]);
    const C T = r.T_ref + n0;
    const C q1 = r.om_a * n1 + r.z_a * (ux * T);
    const C q2 = r.om_a * n2 + r.z_a * (uy * T);
    const C q3 = r.om_ze * n3 + r.zv_e * n0;
    const C q4 = r.om_zn * n4;
    const C c3 = C(0.25) * q3, c4 = C(0.25) * q4;
    t[0] = n0 - q3;
    t[1] = (c3 + c4) + C(0.5) * q1;
    t[3] = (c3 + c4) - C(0.5) * q1;
    t[2] = (c3 - c4) + C(0.5) * q2;
    t[4] = (c3 - c4) - C(0.5) * q2;
    }
}

// ------------------------------------------- FP32 collision, explicit rounding

// Correctly rounded FP32 operations on one value (float) or on a pair of
// values in one packed instruction (float2, the sm_100+ FFMA2/FADD2/FMUL2
// path). The FP32/FP16 kernels all collide through collide_x, either per cell
// or per pair of cells, with the same sequence of operations, so every kernel
// variant produces the same bits.
template <typename T>
struct Ops;

template <>
struct Ops<float> {
    using V = float;
    static __device__ __forceinline__ float bc(float c) { return c; }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fadd_rn(a, -b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};

template <>
struct Ops<float2> {
    using V = float;
    static __device__ __forceinline__ float2 bc(float c) { return make_float2(c, c); }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    // a - b as fma(b, -1, a): one rounding of the exact difference
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) {
        return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
    }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
};

template <>
struct Ops<double> {
    using V = double;
    static __device__ __forceinline__ double bc(double c) { return c; }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// thermal_q9 with every rounding explicit (T is float or float2).
template <typename T>
__device__ __forceinline__ void thermal_q9_x(const RatesC<float> &r, T t[9], T n0, T ux, T uy, T uu) {
    using O = Ops<T>;
    const T b13 = O::add(t[1], t[3]), e13 = O::sub(t[1], t[3]);
    const T b24 = O::add(t[2], t[4]), e24 = O::sub(t[2], t[4]);
    const T b57 = O::add(t[5], t[7]), e57 = O::sub(t[5], t[7]);
    const T b68 = O::add(t[6], t[8]), e68 = O::sub(t[6], t[8]);
    const T Dt = O::add(b57, b68);
    const T n6 = O::add(e57, e68), n7 = O::sub(e57, e68);
    const T n1 = O::add(e13, n7), n2 = O::add(e24, n6);
    const T n3 = O::add(O::add(b13, b24), O::add(Dt, Dt));
    const T n4 = O::sub(b13, b24), n5 = O::sub(b57, b68);
    const T Tm = O::add(O::bc(r.T_ref), n0);
    const T Tuu = O::mul(O::bc(r.theta), O::mul(Tm, uu));
    const T q1 = O::fma(O::bc(r.om_a), n1, O::mul(O::bc(r.z_a), O::mul(Tm, ux)));
    const T q2 = O::fma(O::bc(r.om_a), n2, O::mul(O::bc(r.z_a), O::mul(Tm, uy)));
    const T q3 = O::fma(O::bc(r.om_ze), n3, O::mul(O::bc(r.z_e), O::fma(O::bc(2.0f / 3.0f), n0, Tuu)));
    const T dxy = O::fma(ux, ux, O::mul(O::bc(-1.f), O::mul(uy, uy)));
    const T q4 = O::fma(O::bc(r.om_zn), n4, O::mul(O::bc(r.z_nu), O::mul(O::bc(r.theta), O::mul(Tm, dxy))));
    const T q5 = O::fma(O::bc(r.om_zn), n5, O::mul(O::bc(r.z_nu), O::mul(O::bc(r.theta), O::mul(Tm, O::mul(ux, uy)))));
    const T q6 = O::fma(O::bc(r.om_zq), n6, O::mul(O::bc(r.z_q), O::mul(O::bc(1.0f / 3.0f), O::mul(Tm, uy))));
    const T q7 = O::fma(O::bc(r.om_zq), n7, O::mul(O::bc(r.z_q), O::mul(O::bc(1.0f / 3.0f), O::mul(Tm, ux))));
    const T q8 = O::fma(O::bc(r.om_zeps), Dt,
                        O::mul(O::bc(r.z_eps), O::fma(O::bc(1.0f / 9.0f), n0, O::mul(O::bc(1.0f / 3.0f), Tuu))));
    const T A = O::fma(O::bc(0.25f), q3, O::mul(O::bc(-0.5f), q8));
    const T B = O::mul(O::bc(0.25f), q4);
    const T h1 = O::mul(O::bc(0.5f), O::sub(q1, q7));
    const T h2 = O::mul(O::bc(0.5f), O::sub(q2, q6));
    const T P = O::mul(O::bc(0.25f), O::add(q8, q5));
    const T Q = O::mul(O::bc(0.25f), O::add(q6, q7));
    const T R = O::mul(O::bc(0.25f), O::sub(q8, q5));
    const T Sx = O::mul(O::bc(0.25f), O::sub(q6, q7));
    const T AB = O::add(A, B), AmB = O::sub(A, B);
    t[0] = O::add(O::sub(n0, q3), q8);
    t[1] = O::add(AB, h1);
    t[3] = O::sub(AB, h1);
    t[2] = O::add(AmB, h2);
    t[4] = O::sub(AmB, h2);
    t[5] = O::add(P, Q);
    t[7] = O::sub(P, Q);
    t[6] = O::add(R, Sx);
    t[8] = O::sub(R, Sx);
}

// Same method as collide<float> (Eq. 8 with Eqs. 16, 17, 20; Eq. 24 with
// Eqs. 28, 29; M and M^-1 of Eqs. 13 and A1 on pair sums), every rounding
// explicit. T is float (one cell) or float2 (two cells).
template <typename T, int TQ = 5>
__device__ __forceinline__ void collide_x(const RatesC<float> &r, T f[9], T t[TQ]) {
    using O = Ops<T>;
    T n0;
    if constexpr (TQ == 9)
        n0 = O::add(O::add(O::add(O::add(t[0], t[1]), O::add(t[2], t[3])), O::add(t[4], t[5])),
                    O::add(O::add(t[6], t[7]), t[8]));
    else
        n0 = O::add(O::add(O::add(t[0], t[1]), O::add(t[2], t[3])), t[4]);  // T - T_ref
    const T Fx = O::bc(r.ax);
    const T Fy = O::fma(O::bc(r.g_beta), n0, O::bc(r.Fy0));  // Eq. 4
    // D2Q9 forward map (Eq. 13)
    const T a13 = O::add(f[1], f[3]), d13 = O::sub(f[1], f[3]);
    const T a24 = O::add(f[2], f[4]), d24 = O::sub(f[2], f[4]);
    const T a57 = O::add(f[5], f[7]), d57 = O::sub(f[5], f[7]);
    const T a68 = O::add(f[6], f[8]), d68 = O::sub(f[6], f[8]);
    const T D = O::add(a57, a68);
    const T A4 = O::add(a13, a24);
    const T m0 = O::add(O::add(f[0], A4), D);
    const T m6 = O::add(d57, d68);
    const T m7 = O::sub(d57, d68);
    const T jx = O::add(d13, m7);
    const T jy = O::add(d24, m6);
    const T m3 = O::add(A4, O::add(D, D));
    const T m4 = O::sub(a13, a24);
    const T m5 = O::sub(a57, a68);
    // Eq. 19 with rho0 = 1
    const T ux = O::add(jx, O::bc(r.hx));
    const T uy = O::fma(O::bc(0.5f), Fy, jy);
    const T uyuy = O::mul(uy, uy);
    const T uu = O::fma(ux, ux, uyuy);
    const T uF = O::fma(ux, Fx, O::mul(uy, Fy));
    // Eq. 8
    const T p1 = O::add(jx, Fx);
    const T p2 = O::add(jy, Fy);
    const T p3 = O::fma(O::bc(r.om_e), m3,
                        O::fma(O::bc(r.s_e), O::fma(O::bc(2.0f / 3.0f), m0, uu), O::mul(O::bc(r.h2e), uF)));
    const T dxy = O::fma(ux, ux, O::mul(O::bc(-1.f), uyuy));
    const T dF = O::fma(ux, Fx, O::mul(O::bc(-1.f), O::mul(uy, Fy)));
    const T p4 = O::fma(O::bc(r.om_nu), m4, O::fma(O::bc(r.s_nu), dxy, O::mul(O::bc(r.h2nu), dF)));
    const T cF = O::fma(ux, Fy, O::mul(uy, Fx));
    const T p5 = O::fma(O::bc(r.om_nu), m5, O::fma(O::bc(r.s_nu), O::mul(ux, uy), O::mul(O::bc(r.h_nu), cF)));
    const T p6 = O::fma(O::bc(r.om_q), m6, O::mul(O::bc(1.0f / 3.0f), O::fma(O::bc(r.s_q), jy, Fy)));
    const T p7 = O::fma(O::bc(r.om_q), m7, O::mul(O::bc(1.0f / 3.0f), O::fma(O::bc(r.s_q), jx, Fx)));
    const T p8 = O::fma(O::bc(r.om_eps), D,
                        O::fma(O::bc(r.s_eps), O::fma(O::bc(1.0f / 9.0f), m0, O::mul(O::bc(1.0f / 3.0f), uu)),
                               O::mul(O::bc(r.h23eps), uF)));
    // back map (Eq. A1); the 1/2 and 1/4 scalings are exact
    const T A = O::fma(O::bc(0.25f), p3, O::mul(O::bc(-0.5f), p8));
    const T B = O::mul(O::bc(0.25f), p4);
    const T h1 = O::mul(O::bc(0.5f), O::sub(p1, p7));
    const T h2 = O::mul(O::bc(0.5f), O::sub(p2, p6));
    const T P = O::mul(O::bc(0.25f), O::add(p8, p5));
    const T Q = O::mul(O::bc(0.25f), O::add(p6, p7));
    const T R = O::mul(O::bc(0.25f), O::sub(p8, p5));
    const T Sx = O::mul(O::bc(0.25f), O::sub(p6, p7));
    const T AB = O::add(A, B), AmB = O::sub(A, B);
    f[0] = O::add(O::sub(m0, p3), p8);
    f[1] = O::add(AB, h1);
    f[3] = O::sub(AB, h1);
    f[2] = O::add(AmB, h2);
    f[4] = O::sub(AmB, h2);
    f[5] = O::add(P, Q);
    f[7] = O::sub(P, Q);
    f[6] = O::add(R, Sx);
    f[8] = O::sub(R, Sx);
    if constexpr (TQ == 9) {
        thermal_q9_x<T>(r, t, n0, ux, uy, uu);
        return;
    } else {
    // D2Q5 forward map (Eq. 26), relaxation (Eq. 24) and back map (Eq. A2)
    const T s13 = O::add(t[1], t[3]), s24 = O::add(t[2], t[4]);
    const T n1 = O::sub(t[1], t[3]);
    const T n2 = O::sub(t[2], t[4]);
    const T n3 = O::add(s13, s24);
    const T n4 = O::sub(s13, s24);
    const T Tm = O::add(O::bc(r.T_ref), n0);
    const T q1 = O::fma(O::bc(r.om_a), n1, O::mul(O::bc(r.z_a), O::mul(ux, Tm)));
    const T q2 = O::fma(O::bc(r.om_a), n2, O::mul(O::bc(r.z_a), O::mul(uy, Tm)));
    const T q3 = O::fma(O::bc(r.om_ze), n3, O::mul(O::bc(r.zv_e), n0));
    const T q4 = O::mul(O::bc(r.om_zn), n4);
    const T c3 = O::mul(O::bc(0.25f), q3), c4 = O::mul(O::bc(0.25f), q4);
    const T c34 = O::add(c3, c4), c3m4 = O::sub(c3, c4);
    t[0] = O::sub(n0, q3);
    t[1] = O::fma(O::bc(0.5f), q1, c34);
    t[3] = O::fma(O::bc(-0.5f), q1, c34);
    t[2] = O::fma(O::bc(0.5f), q2, c3m4);
    t[4] = O::fma(O::bc(-0.5f), q2, c3m4);
    }
}

// ------------------------------------------------------------ BGK collision

// e_I . (x, y) for the D2Q9 velocities of Eq. 5 (I >= 1), exactly.
template <int I, typename O, typename T>
__device__ __forceinline__ T edot(T x, T y) {
    if constexpr (I == 1) return x;
    else if constexpr (I == 2) return y;
    else if constexpr (I == 3) return O::mul(O::bc(-1), x);
    else if constexpr (I == 4) return O::mul(O::bc(-1), y);
    else if constexpr (I == 5) return O::add(x, y);
    else if constexpr (I == 6) return O::sub(y, x);
    else if constexpr (I == 7) return O::mul(O::bc(-1), O::add(x, y));
    else return O::sub(x, y);
}

// Directions I and J = opp(I) of the BGK collision (see collide_bgk_x). Both
// equilibria and forcing terms split into a part even in e (shared) and a part
// odd in e (sign flipped): with eu = e_I.u, eF = e_I.F and C0 = s base - 3 h u.F,
//   f*_I,J = (1 - s) f_I,J + w [C0 + eu (4.5 s eu + 9 h eF)] +- 3 w (s eu + h eF).
template <int I, int J, typename T, typename R, int TQ>
__device__ __forceinline__ void bgk_pair(const R &r, T f[9], T t[TQ], T C0, T ux, T uy, T Fx, T Fy, T uu, T zn0,
                                         T zT) {
    using O = Ops<T>;
    using V = typename O::V;
    constexpr double w = I < 5 ? 1.0 / 9 : 1.0 / 36;
    const T W = O::bc((V)w), W3 = O::bc((V)(3.0 * w));
    const T eu = edot<I, O>(ux, uy), eF = edot<I, O>(Fx, Fy);
    const T hF = O::mul(O::bc(r.h_nu), eF);
    const T ev = O::mul(W, O::fma(eu, O::fma(O::mul(O::bc((V)4.5), O::bc(r.s_nu)), eu, O::mul(O::bc(9), hF)), C0));
    const T od = O::mul(W3, O::fma(O::bc(r.s_nu), eu, hF));
    f[I] = O::fma(O::bc(r.om_nu), f[I], O::add(ev, od));
    f[J] = O::fma(O::bc(r.om_nu), f[J], O::sub(ev, od));
    if constexpr (TQ == 9 || J < 5) {
        T evT, odT;
        if constexpr (TQ == 9) {
            // zeta w [(T - T_ref) + T theta (4.5 eu^2 - 1.5 u^2)] +- 3 zeta w T eu  (Eq. 31, storage frame)
            const T q2 = O::fma(O::mul(O::bc((V)4.5), eu), eu, O::mul(O::bc((V)-1.5), uu));
            evT = O::mul(W, O::fma(O::mul(zT, O::bc(r.theta)), q2, zn0));
            odT = O::mul(W3, O::mul(zT, eu));
        } else {
            // zeta [(varpi/4)(T - T_ref)] +- zeta (1/2) T eu  (Eq. 30, storage frame)
            evT = O::mul(O::mul(O::bc((V)0.25), O::bc(r.varpi)), zn0);
            odT = O::mul(O::bc((V)0.5), O::mul(zT, eu));
        }
        t[I] = O::fma(O::bc(r.om_a), t[I], O::add(evT, odT));
        t[J] = O::fma(O::bc(r.om_a), t[J], O::sub(evT, odT));
    }
}

// BGK: the special case of Eqs. 8 and 24 (or Eq. 32) with one rate for the
// flow (s = s_nu, h = 1 - s/2) and one for temperature (zeta = zeta_alpha),
// written in velocity space, every rounding explicit (T = double, float or
// float2; R = RatesC of its scalar type):
//   f*_i = f_i - s (f_i - f_eq_i) + h w_i [3 (e_i - u) . F + 9 (e_i . u)(e_i . F)]
//   g*_i = g_i - zeta (g_i - g_eq_i)
// with the incompressible equilibrium f_eq_i = w_i [rho + 3 e_i.u + 4.5 (e_i.u)^2
// - 1.5 u^2] (rho0 = 1), the forcing term of Guo, Zheng and Shi (Phys. Rev. E 65,
// 046308, 2002), and g_eq of Eq. 30 (D2Q5) or Eq. 31 (D2Q9). In the storage frame
// every equilibrium is shifted like the populations. Opposite directions are
// updated together (bgk_pair).
template <typename T, typename R, int TQ>
__device__ __forceinline__ void collide_bgk_x(const R &r, T f[9], T t[TQ]) {
    using O = Ops<T>;
    using V = typename O::V;
    T n0;
    if constexpr (TQ == 9)
        n0 = O::add(O::add(O::add(O::add(t[0], t[1]), O::add(t[2], t[3])), O::add(t[4], t[5])),
                    O::add(O::add(t[6], t[7]), t[8]));
    else
        n0 = O::add(O::add(O::add(t[0], t[1]), O::add(t[2], t[3])), t[4]);
    const T Fx = O::bc(r.ax);
    const T Fy = O::fma(O::bc(r.g_beta), n0, O::bc(r.Fy0));  // Eq. 4
    const T a13 = O::add(f[1], f[3]), d13 = O::sub(f[1], f[3]);
    const T a24 = O::add(f[2], f[4]), d24 = O::sub(f[2], f[4]);
    const T a57 = O::add(f[5], f[7]), d57 = O::sub(f[5], f[7]);
    const T a68 = O::add(f[6], f[8]), d68 = O::sub(f[6], f[8]);
    const T m0 = O::add(O::add(f[0], O::add(a13, a24)), O::add(a57, a68));  // Eq. 18
    const T jx = O::add(d13, O::sub(d57, d68));
    const T jy = O::add(d24, O::add(d57, d68));
    const T ux = O::add(jx, O::bc(r.hx));  // Eq. 19, rho0 = 1
    const T uy = O::fma(O::bc((V)0.5), Fy, jy);
    const T uu = O::fma(ux, ux, O::mul(uy, uy));
    const T uF = O::fma(ux, Fx, O::mul(uy, Fy));
    // C0 = s (rho - 1.5 u^2) - 3 h u.F, the isotropic part of s f_eq / w + h F / w
    const T C0 = O::fma(O::bc(r.s_nu), O::fma(O::bc((V)-1.5), uu, m0), O::mul(O::mul(O::bc(-3), O::bc(r.h_nu)), uF));
    const T Tm = O::add(O::bc(r.T_ref), n0);
    const T zn0 = O::mul(O::bc(r.z_a), n0), zT = O::mul(O::bc(r.z_a), Tm);
    f[0] = O::fma(O::bc(r.om_nu), f[0], O::mul(O::bc((V)(4.0 / 9)), C0));
    if constexpr (TQ == 9) {
        // zeta (4/9) [(T - T_ref) - 1.5 theta T u^2]
        const T q2 = O::mul(O::bc((V)-1.5), uu);
        t[0] = O::fma(O::bc(r.om_a), t[0], O::mul(O::bc((V)(4.0 / 9)), O::fma(O::mul(zT, O::bc(r.theta)), q2, zn0)));
    } else {
        t[0] = O::fma(O::bc(r.om_a), t[0], O::mul(O::sub(O::bc(1), O::bc(r.varpi)), zn0));
    }
    bgk_pair<1, 3, T, R, TQ>(r, f, t, C0, ux, uy, Fx, Fy, uu, zn0, zT);
    bgk_pair<2, 4, T, R, TQ>(r, f, t, C0, ux, uy, Fx, Fy, uu, zn0, zT);
    bgk_pair<5, 7, T, R, TQ>(r, f, t, C0, ux, uy, Fx, Fy, uu, zn0, zT);
    bgk_pair<6, 8, T, R, TQ>(r, f, t, C0, ux, uy, Fx, Fy, uu, zn0, zT);
}

// The collision of one cell in the storage's compute type: MRT (exact FP64
// operators, or explicit FP32 rounding for shifted storage) or BGK.
template <typename S, int TQ, bool BGK>
__device__ __forceinline__ void collide_cell(const RatesC<typename Store<S>::C> &r, typename Store<S>::C f[9],
                                             typename Store<S>::C t[TQ]) {
    using C = typename Store<S>::C;
    if constexpr (BGK) collide_bgk_x<C, RatesC<C>, TQ>(r, f, t);
    else if constexpr (Store<S>::kShifted) collide_x<float, TQ>(r, f, t);
    else collide<C, TQ>(r, f, t);
}

// Collide cells K and K + 1 of an N-cell group as one float2 pair, in place.
template <int K, int N, int TQ = 5, bool BGK = false>
__device__ __forceinline__ void collide_pair(const RatesC<float> &r, float f[9][N], float t[TQ][N]) {
    float2 fp[9], tp[TQ];
#pragma unroll
    for (int i = 0; i < 9; ++i) fp[i] = make_float2(f[i][K], f[i][K + 1]);
#pragma unroll
    for (int i = 0; i < TQ; ++i) tp[i] = make_float2(t[i][K], t[i][K + 1]);
    if constexpr (BGK) collide_bgk_x<float2, RatesC<float>, TQ>(r, fp, tp);
    else collide_x<float2, TQ>(r, fp, tp);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        f[i][K] = fp[i].x;
        f[i][K + 1] = fp[i].y;
    }
#pragma unroll
    for (int i = 0; i < TQ; ++i) {
        t[i][K] = tp[i].x;
        t[i][K + 1] = tp[i].y;
    }
}

// Halfway wall links of cell K of an N-cell group (link-map bytes mN), in place.
template <typename S, int K, int N, typename PA, bool NC = true, int TQ = 5>
__device__ __forceinline__ void wall_links(const PA &pl, const Geom &g, uint32_t mN, int x0, int r0, int rm,
                                           int rp, float f[9][N], float t[TQ][N]) {
    const unsigned m = (mN >> (8 * K)) & 0xFFu;
    if (m == 0 || m == kSolid) return;
    const int x = x0 + K;
    int xm = x - 1, xp = x + 1;
    if (g.px) {
        xm = (xm < 0) ? xm + g.nx : xm;
        xp = (xp >= g.nx) ? xp - g.nx : xp;
    }
    const int sidx[9] = {r0 + x, r0 + xm, rm + x, r0 + xp, rp + x, rm + xm, rm + xp, rp + xp, rp + xm};
    const int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (m & (1u << (i - 1))) {
            const WallDev *w = wall_of(g, sidx[i], 22);
            if (kBoundsBuild && !w) continue;
            const S *pf = pl.src_at(opp[i]) + r0 + x;
            f[i][K] = (NOMRT_OK(g, pf, sizeof(S), 23) ? Ld<S, NC>::one(pf) : 0.f) + (float)__ldg(&w->cf[i]);
            if (i < TQ) {
                const S *pt = pl.src_at(9 + opp[i]) + r0 + x;
                t[i][K] = (float)__ldg(&w->tsgn) * (NOMRT_OK(g, pt, sizeof(S), 24) ? Ld<S, NC>::one(pt) : 0.f) +
                          (float)__ldg(TQ == 9 ? &w->tb9[i] : &w->tb);
            }
        }
    }
}

// Solid cell K of a group: write zeros (solid cells hold zeros).
template <int K, int N, int TQ = 5>
__device__ __forceinline__ void zero_solid(uint32_t mN, float f[9][N], float t[TQ][N]) {
    if (((mN >> (8 * K)) & 0xFFu) != kSolid) return;
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i][K] = 0.f;
#pragma unroll
    for (int i = 0; i < TQ; ++i) t[i][K] = 0.f;
}

// ------------------------------------------------------------------ kernels

template <typename S, int TQ = 5, bool BGK = false>
__global__ void __launch_bounds__(256) k_step(const Planes<S> pl, const Geom g, const RatesC<typename Store<S>::C> r) {
    using C = typename Store<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.nx) return;
    for (int y = blockIdx.y * blockDim.y + threadIdx.y; y < g.ny; y += gridDim.y * blockDim.y) {
        const int off = y * g.pitch + x;
        const unsigned m = NOMRT_OK(g, g.mask + off, 1, 6) ? __ldg(g.mask + off) : (unsigned)kSolid;
        if (m == kSolid) continue;
        C f[9], t[TQ];
        pull<S, TQ>(pl.src, g, x, y, m, f, t);
        collide_cell<S, TQ, BGK>(r, f, t);
#pragma unroll
        for (int q = 0; q < 9; ++q)
            if (NOMRT_OK(g, pl.dst[q] + off, sizeof(S), 7)) Store<S>::st(pl.dst[q] + off, f[q]);
#pragma unroll
        for (int q = 0; q < TQ; ++q)
            if (NOMRT_OK(g, pl.dst[9 + q] + off, sizeof(S), 7)) Store<S>::st(pl.dst[9 + q] + off, t[q]);
    }
}

// Boundary nodes of NEE walls: rebuild (non-equilibrium extrapolation), collide,
// store. Runs after a step kernel that skipped them (their link-map byte is
// kSolid), reading the same source buffer.
template <typename S, int TQ = 5, bool BGK = false>
__global__ void __launch_bounds__(128) k_nee(const Planes<S> pl, const Geom g, const RatesC<typename Store<S>::C> r,
                                             const int2 *nee, int n) {
    using C = typename Store<S>::C;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!NOMRT_OK(g, nee + i, sizeof(int2), 25)) return;
    const int2 e = nee[i];
    const int off = e.x, d = e.y & 0xFF, k = e.y >> 8;
    const int y = off / g.pitch, x = off - y * g.pitch;
    if (!NOMRT_OK(g, g.walls + k, sizeof(WallDev), 26)) return;
    C f[9], t[TQ];
    nee_rebuild<S, TQ>(pl.src, g, r, x, y, d, g.walls + k, f, t);
    collide_cell<S, TQ, BGK>(r, f, t);
#pragma unroll
    for (int q = 0; q < 9; ++q)
        if (NOMRT_OK(g, pl.dst[q] + off, sizeof(S), 27)) Store<S>::st(pl.dst[q] + off, f[q]);
#pragma unroll
    for (int q = 0; q < TQ; ++q)
        if (NOMRT_OK(g, pl.dst[9 + q] + off, sizeof(S), 27)) Store<S>::st(pl.dst[9 + q] + off, t[q]);
}

// Initial state (rest equilibrium, Eqs. 22, 30 at u = 0) in the storage frame.
// The temperature weights of the storage frame: D2Q5 (Eq. 30 at u = 0, with
// varpi of Eq. 28) or the D2Q9 weights (Eq. 31 at u = 0).
__device__ __forceinline__ double thermal_weight(int q, int tq, double varpi) {
    if (tq == 9) return q == 0 ? 4.0 / 9 : (q < 5 ? 1.0 / 9 : 1.0 / 36);
    return q == 0 ? 1.0 - varpi : 0.25 * varpi;
}

// Rows [r0, r1) of the initial state into the source buffer (every column of
// the pitched rows: solid cells and padding get zeros), and zeros into the
// other buffer. T: rows r0.. of the initial temperature (nx per row), or
// nullptr for T0 everywhere.
template <typename S>
__global__ void k_init_rows(const Planes<S> pl, const Geom g, int r0, int r1, const double *T, double T0,
                            double T_ref, double varpi, int shifted, int tq) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = r0 + blockIdx.y;
    if (x >= g.pitch || y >= r1) return;
    const int off = y * g.pitch + x;
    const bool fluid = x < g.nx && kept_cell(g, off);
    const double w9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const double Tn = fluid ? (T ? T[(size_t)(y - r0) * g.nx + x] : T0) : 0.0;
    for (int q = 0; q < 9; ++q) {
        double v = fluid ? (shifted ? 0.0 : w9[q]) : 0.0;
        Store<S>::st(const_cast<S *>(pl.src[q]) + off, (typename Store<S>::C)v);
        Store<S>::st(pl.dst[q] + off, (typename Store<S>::C)0.0);
    }
    for (int q = 0; q < tq; ++q) {
        const double wT = thermal_weight(q, tq, varpi);
        double v = fluid ? wT * (Tn - T_ref) : 0.0;
        Store<S>::st(const_cast<S *>(pl.src[9 + q]) + off, (typename Store<S>::C)v);
        Store<S>::st(pl.dst[9 + q] + off, (typename Store<S>::C)0.0);
    }
}

// rho, u_x, u_y, T of rows [r0, r1) into out[0..3] (each (r1 - r0) * nx
// doubles, row y at (y - r0) * nx; a NULL output is skipped). The outputs may
// be a staging area or the caller's page-locked host arrays.
template <typename S, int TQ = 5>
__global__ void k_macro_rows(const Planes<S> pl, const Geom g, const RatesC<typename Store<S>::C> r, int r0,
                             int r1, double rho_ref, double T_ref, double *o_rho, double *o_ux, double *o_uy,
                             double *o_T) {
    using C = typename Store<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = r0 + blockIdx.y;
    if (x >= g.nx || y >= r1) return;
    const size_t o = (size_t)(y - r0) * g.nx + x;
    const unsigned m = g.mask[y * g.pitch + x];
    const unsigned d = g.nee_dir[y * g.pitch + x];
    double v[4] = {0, 0, 0, 0};
    if (m != kSolid || d != 0) {
        C f[9], t[TQ];
        if (m != kSolid) pull<S, TQ>(pl.src, g, x, y, m, f, t);
        else nee_rebuild<S, TQ>(pl.src, g, r, x, y, (int)d, g.walls + g.flags[y * g.pitch + x], f, t);
        Macro<C> M = macro_of<C, TQ>(r, f, t);
        v[0] = rho_ref + (double)M.drho;
        v[1] = (double)M.ux;
        v[2] = (double)M.uy;
        v[3] = T_ref + (double)M.dT;
    }
    if (o_rho) o_rho[o] = v[0];
    if (o_ux) o_ux[o] = v[1];
    if (o_uy) o_uy[o] = v[2];
    if (o_T) o_T[o] = v[3];
}

template <typename S>
__global__ void k_export_rows(const Planes<S> pl, const Geom g, int r0, int r1, double rho_ref, double T_ref,
                              double varpi, int tq, double *out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = r0 + blockIdx.y;
    if (x >= g.nx || y >= r1) return;
    const size_t n = (size_t)(r1 - r0) * g.nx;
    const size_t o = (size_t)(y - r0) * g.nx + x;
    const int off = y * g.pitch + x;
    const bool fluid = kept_cell(g, off);
    const double w9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    for (int q = 0; q < 9 + tq; ++q) {
        double v = 0.0;
        if (fluid) {
            double shift = q < 9 ? w9[q] * rho_ref : thermal_weight(q - 9, tq, varpi) * T_ref;
            v = (double)Store<S>::ld(pl.src[q] + off) + shift;
        }
        out[q * n + o] = v;
    }
}

// which: bit 0 = f planes present, bit 1 = g planes present
template <typename S>
__global__ void k_import_rows(const Planes<S> pl, const Geom g, int r0, int r1, double rho_ref, double T_ref,
                              double varpi, int tq, const double *in, int which) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = r0 + blockIdx.y;
    if (x >= g.nx || y >= r1) return;
    const size_t n = (size_t)(r1 - r0) * g.nx;
    const size_t o = (size_t)(y - r0) * g.nx + x;
    const int off = y * g.pitch + x;
    const bool fluid = kept_cell(g, off);
    const double w9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    for (int q = 0; q < 9 + tq; ++q) {
        if (q < 9 && !(which & 1)) continue;
        if (q >= 9 && !(which & 2)) continue;
        double shift = q < 9 ? w9[q] * rho_ref : thermal_weight(q - 9, tq, varpi) * T_ref;
        double v = fluid ? in[q * n + o] - shift : 0.0;
        Store<S>::st(const_cast<S *>(pl.src[q]) + off, (typename Store<S>::C)v);
    }
}

// ------------------------------------------------------------- reductions

template <int W>
__device__ __forceinline__ void block_reduce_store(double (&v)[W], double *partials) {
    __shared__ double sh[kRedThreads / 32][W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < W; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < W; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
            double a = lane < kRedThreads / 32 ? sh[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) partials[blockIdx.x * W + k] = a;
        }
    }
}

// Temperature after the pull at one fluid cell (Eq. 27; the zeroth moment of
// the D2Q9 model), FP64 accumulation.
template <typename S, int TQ>
__device__ __forceinline__ double temperature_at(const Planes<S> &pl, const Geom &g, int x, int y, double T_ref) {
    using C = typename Store<S>::C;
    const unsigned m = g.mask[y * g.pitch + x];
    C f[9], t[TQ];
    pull<S, TQ>(pl.src, g, x, y, m, f, t);
    double s = ((((double)t[0] + (double)t[1]) + ((double)t[2] + (double)t[3])) + (double)t[4]);
    if constexpr (TQ == 9) s += (((double)t[5] + (double)t[6]) + ((double)t[7] + (double)t[8]));
    return T_ref + s;
}

// Eq. 39 with the one-sided wall gradient; one thread per line along the wall.
template <typename S, int TQ = 5>
__global__ void __launch_bounds__(kRedThreads) k_nusselt(const Planes<S> pl, const Geom g, int side, double L,
                                                         double dT, double T_ref, double *partials) {
    const int along = side < 2 ? g.ny : g.nx;
    double v[2] = {0.0, 0.0};
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < along; s += gridDim.x * blockDim.x) {
        int wx, wy, dx, dy;
        if (side == 0) { wx = 0; wy = s; dx = 1; dy = 0; }
        else if (side == 1) { wx = g.nx - 1; wy = s; dx = -1; dy = 0; }
        else if (side == 2) { wx = s; wy = 0; dx = 0; dy = 1; }
        else { wx = s; wy = g.ny - 1; dx = 0; dy = -1; }
        const int x1 = wx + dx, y1 = wy + dy, x2 = wx + 2 * dx, y2 = wy + 2 * dy;
        if (x2 < 0 || x2 >= g.nx || y2 < 0 || y2 >= g.ny) continue;
        const int k = g.flags[wy * g.pitch + wx];
        if (k == 0) continue;
        if (g.mask[y1 * g.pitch + x1] == kSolid || g.mask[y2 * g.pitch + x2] == kSolid) continue;
        const WallDev *w = g.walls + k;
        if (w->tsgn > 0.0) continue;  // adiabatic: no wall temperature
        const double Tw = w->Tw;
        const double T1 = temperature_at<S, TQ>(pl, g, x1, y1, T_ref);
        const double T2 = temperature_at<S, TQ>(pl, g, x2, y2, T_ref);
        // halfway wall half a cell before c1; node-based wall on the wall node itself
        const double dTds = w->nee != 0.0 ? (-3.0 * Tw + 4.0 * T1 - T2) / 2.0 : (9.0 * T1 - T2 - 8.0 * Tw) / 3.0;
        const double dTdn = (side == 0 || side == 2) ? dTds : -dTds;
        v[0] += -L * dTdn / dT;
        v[1] += 1.0;
    }
    block_reduce_store<2>(v, partials);
}

template <typename S, int TQ = 5>
__global__ void __launch_bounds__(kRedThreads) k_residual(const Planes<S> pl, const Geom g,
                                                          const RatesC<typename Store<S>::C> r, double T_ref,
                                                          double *snap, size_t plane, int have_snap,
                                                          double *partials) {
    using C = typename Store<S>::C;
    double v[5] = {0, 0, 0, 0, 0};
    const long long total = (long long)g.ny * g.nx;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < total;
         c += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(c / g.nx), x = (int)(c - (long long)y * g.nx);
        const int off = y * g.pitch + x;
        const unsigned m = g.mask[off];
        if (m == kSolid) continue;
        C f[9], t[TQ];
        pull<S, TQ>(pl.src, g, x, y, m, f, t);
        Macro<C> M = macro_of<C, TQ>(r, f, t);
        const double ux = (double)M.ux, uy = (double)M.uy, T = T_ref + (double)M.dT;
        if (have_snap) {
            const double a = ux - snap[off], b = uy - snap[plane + off], d = T - snap[2 * plane + off];
            v[0] += a * a + b * b;
            v[2] += d * d;
        }
        v[1] += ux * ux + uy * uy;
        v[3] += T * T;
        if (!isfinite(ux) || !isfinite(uy) || !isfinite(T)) v[4] += 1.0;
        snap[off] = ux;
        snap[plane + off] = uy;
        snap[2 * plane + off] = T;
    }
    block_reduce_store<5>(v, partials);
}

// ------------------------------------------------- vectorised step kernel

// Four compute values -> four consecutive storage elements (128-bit FP32, 64-bit
// FP16 stores), and the shared-memory reads of the staged kernel (loads from
// global memory go through Ld<S, NC>).
template <typename S>
struct Vec4;

template <>
struct Vec4<float> {
    static __device__ __forceinline__ void st(float *p, const float a[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(a[0], a[1], a[2], a[3]);
    }
    static __device__ __forceinline__ void ld_shared(const float *p, float a[4]) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
    }
};

template <>
struct Vec4<__half> {
    static __device__ __forceinline__ void st(__half *p, const float a[4]) {
        const __half2 h0 = __floats2half2_rn(a[0], a[1]), h1 = __floats2half2_rn(a[2], a[3]);
        uint2 v;
        memcpy(&v.x, &h0, 4);
        memcpy(&v.y, &h1, 4);
        *reinterpret_cast<uint2 *>(p) = v;
    }
    static __device__ __forceinline__ void ld_shared(const __half *p, float a[4]) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        __half2 h0, h1;
        memcpy(&h0, &v.x, 4);
        memcpy(&h1, &v.y, 4);
        const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
        a[0] = f0.x; a[1] = f0.y; a[2] = f1.x; a[3] = f1.y;
    }
};

constexpr unsigned kFull = 0xffffffffu;

// The four values of one population plane that cells x0..x0+3 of a row pull.
// DX = +1: a direction with e_x = +1 pulls from x - 1; DX = -1 pulls from
// x + 1. The in-row neighbour comes from the adjacent lane's vector; lanes at
// the warp's edges load it directly, and the periodic seam (x = 0 pulling from
// nx - 1, x = nx - 1 pulling from 0) is loaded directly too. Every lane of the
// warp must call this (shuffles). `inrow` (x0 < pitch) gates the loads, not the
// lane's own fluid cells: a lane of solid cells still supplies its neighbours.
template <typename S, int DX, bool NC = true>
__device__ __forceinline__ void ld_plane(const S *row, const Geom &g, int x0, int lane, bool inrow, float out[4]) {
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    if (inrow && NOMRT_OK(g, row + x0, 4 * sizeof(S), 10)) Ld<S, NC>::four(row + x0, a);
    if (DX == 0) {
        out[0] = a[0]; out[1] = a[1]; out[2] = a[2]; out[3] = a[3];
    } else if (DX == 1) {
        float left = __shfl_up_sync(kFull, a[3], 1);
        if (lane == 0) {
            left = 0.f;
            int xs = x0 - 1;
            if (xs < 0 && g.px) xs += g.nx;
            if (inrow && xs >= 0 && NOMRT_OK(g, row + xs, sizeof(S), 11)) left = Ld<S, NC>::one(row + xs);
        }
        out[0] = left; out[1] = a[0]; out[2] = a[1]; out[3] = a[2];
    } else {
        float right = __shfl_down_sync(kFull, a[0], 1);
        if (lane == 31) {
            right = 0.f;
            const int xs = x0 + 4;
            if (inrow && xs < g.nx && NOMRT_OK(g, row + xs, sizeof(S), 12)) right = Ld<S, NC>::one(row + xs);
        }
        out[0] = a[1]; out[1] = a[2]; out[2] = a[3]; out[3] = right;
        if (g.px && inrow) {
            const int k = g.nx - 1 - x0;
            if (k >= 0 && k < 4) {
                const float v = NOMRT_OK(g, row, sizeof(S), 13) ? Ld<S, NC>::one(row) : 0.f;
#pragma unroll
                for (int j = 0; j < 4; ++j) out[j] = (j == k) ? v : out[j];  // constant indices only
            }
        }
    }
}

// ld_plane without the periodic seam (the caller applies it for all planes at once).
template <typename S, int DX, bool NC = true>
__device__ __forceinline__ void ld_plane_ns(const S *row, const Geom &g, int x0, int lane, bool inrow, float out[4]) {
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    if (inrow && NOMRT_OK(g, row + x0, 4 * sizeof(S), 10)) Ld<S, NC>::four(row + x0, a);
    if (DX == 0) {
        out[0] = a[0]; out[1] = a[1]; out[2] = a[2]; out[3] = a[3];
    } else if (DX == 1) {
        float left = __shfl_up_sync(kFull, a[3], 1);
        if (lane == 0) {
            left = 0.f;
            int xs = x0 - 1;
            if (xs < 0 && g.px) xs += g.nx;
            if (inrow && xs >= 0 && NOMRT_OK(g, row + xs, sizeof(S), 11)) left = Ld<S, NC>::one(row + xs);
        }
        out[0] = left; out[1] = a[0]; out[2] = a[1]; out[3] = a[2];
    } else {
        float right = __shfl_down_sync(kFull, a[0], 1);
        if (lane == 31) {
            right = 0.f;
            const int xs = x0 + 4;
            if (inrow && xs < g.nx && NOMRT_OK(g, row + xs, sizeof(S), 12)) right = Ld<S, NC>::one(row + xs);
        }
        out[0] = a[1]; out[1] = a[2]; out[2] = a[3]; out[3] = right;
    }
}

// Four consecutive values of one population plane (x0..x0+3 of a row), zeros
// where the lane lies past the row (`inrow` false: such a lane still takes part
// in the shuffles that supply its neighbours).
template <typename S, bool NC = true>
__device__ __forceinline__ void ld_four(const Geom &g, const S *row, int x0, bool inrow, float a[4]) {
    a[0] = a[1] = a[2] = a[3] = 0.f;
    if (inrow && NOMRT_OK(g, row + x0, 4 * sizeof(S), 14)) Ld<S, NC>::four(row + x0, a);
}

// The values cells x0..x0+3 pull from a plane with e_x = +1 (source x - 1): the
// left neighbour comes from the previous lane's vector, lane 0 takes `edge`
// (loaded apart, zero where there is none). Every lane of the warp must call it.
__device__ __forceinline__ void pull_from_left(const float a[4], float edge, int lane, float out[4]) {
    float left = __shfl_up_sync(kFull, a[3], 1);
    left = lane == 0 ? edge : left;
    out[0] = left; out[1] = a[0]; out[2] = a[1]; out[3] = a[2];
}

// The same for e_x = -1 (source x + 1): lane 31 takes `edge`; on a periodic x
// the cell nx - 1 (index seam_k of this lane's four, or -1) pulls cell 0's
// value `seam`.
__device__ __forceinline__ void pull_from_right(const float a[4], float edge, int lane, int seam_k, float seam,
                                                float out[4]) {
    float right = __shfl_down_sync(kFull, a[0], 1);
    right = lane == 31 ? edge : right;
    out[0] = a[1]; out[1] = a[2]; out[2] = a[3]; out[3] = right;
#pragma unroll
    for (int j = 0; j < 4; ++j) out[j] = (j == seam_k) ? seam : out[j];  // constant indices only
}

// Fused step, four cells of one row per thread. Same arithmetic as k_step;
// solid cells in a group are written as zeros (they hold zeros already).
// One warp's share of a row: cells x0..x0+3 of row y for each lane (x0 = base +
// 4 lane). Every lane of the warp calls it with the same y. PA gives the plane
// pointers (Planes, or a batch member's).
template <typename S, typename PA, bool NC = true, int TQ = 5, bool BGK = false>
__device__ __forceinline__ void row4(const PA &pl, const Geom &g, const RatesC<float> &r, int x0, int y, int lane) {
    const int r0 = y * g.pitch;
    const bool inrow = x0 < g.pitch;
    uint32_t m4 = 0xFFFFFFFFu;
    if (inrow && NOMRT_OK(g, g.mask + r0 + x0, 4, 15)) m4 = __ldg(reinterpret_cast<const uint32_t *>(g.mask + r0 + x0));
    const bool any = m4 != 0xFFFFFFFFu;
    if (!__any_sync(kFull, any)) return;
    int ym = y - 1, yp = y + 1;
    if (g.py) {
        ym = (ym < 0) ? ym + g.ny : ym;
        yp = (yp >= g.ny) ? yp - g.ny : yp;
    }
    // rows of a non-periodic edge hold no fluid cell, so a warp that gets here has 0 < y < ny - 1
    const int rm = ym * g.pitch, rp = yp * g.pitch;
    float f[9][4], t[TQ][4];
    if constexpr (sizeof(S) == 2) {
        // FP16: each shifted plane loads its own warp-edge values (measured faster for 16-bit
        // storage than the batched form below, which FP32 prefers); the seam is batched
        ld_plane<S, 0, NC>(pl.src_at(0) + r0, g, x0, lane, inrow, f[0]);
        ld_plane<S, 1, NC>(pl.src_at(1) + r0, g, x0, lane, inrow, f[1]);
        ld_plane<S, 0, NC>(pl.src_at(2) + rm, g, x0, lane, inrow, f[2]);
        ld_plane_ns<S, -1, NC>(pl.src_at(3) + r0, g, x0, lane, inrow, f[3]);
        ld_plane<S, 0, NC>(pl.src_at(4) + rp, g, x0, lane, inrow, f[4]);
        ld_plane<S, 1, NC>(pl.src_at(5) + rm, g, x0, lane, inrow, f[5]);
        ld_plane_ns<S, -1, NC>(pl.src_at(6) + rm, g, x0, lane, inrow, f[6]);
        ld_plane_ns<S, -1, NC>(pl.src_at(7) + rp, g, x0, lane, inrow, f[7]);
        ld_plane<S, 1, NC>(pl.src_at(8) + rp, g, x0, lane, inrow, f[8]);
        ld_plane<S, 0, NC>(pl.src_at(9) + r0, g, x0, lane, inrow, t[0]);
        ld_plane<S, 1, NC>(pl.src_at(10) + r0, g, x0, lane, inrow, t[1]);
        ld_plane<S, 0, NC>(pl.src_at(11) + rm, g, x0, lane, inrow, t[2]);
        ld_plane_ns<S, -1, NC>(pl.src_at(12) + r0, g, x0, lane, inrow, t[3]);
        ld_plane<S, 0, NC>(pl.src_at(13) + rp, g, x0, lane, inrow, t[4]);
        if constexpr (TQ == 9) {
            ld_plane<S, 1, NC>(pl.src_at(14) + rm, g, x0, lane, inrow, t[5]);
            ld_plane_ns<S, -1, NC>(pl.src_at(15) + rm, g, x0, lane, inrow, t[6]);
            ld_plane_ns<S, -1, NC>(pl.src_at(16) + rp, g, x0, lane, inrow, t[7]);
            ld_plane<S, 1, NC>(pl.src_at(17) + rp, g, x0, lane, inrow, t[8]);
        }
        {
            // periodic x: the lane holding cell nx - 1 takes cell 0's value of each plane
            // with e_x = -1, in one branch for all of them
            const int kseam = g.nx - 1 - x0;
            if (g.px && inrow && kseam >= 0 && kseam < 4) {
#define NOMRT_SEAM(P, ROW) { const float v = NOMRT_OK(g, ROW, sizeof(S), 16) ? Ld<S, NC>::one(ROW) : 0.f; _Pragma("unroll") for (int j = 0; j < 4; ++j) P[j] = (j == kseam) ? v : P[j]; }
                NOMRT_SEAM(f[3], pl.src_at(3) + r0);
                NOMRT_SEAM(f[6], pl.src_at(6) + rm);
                NOMRT_SEAM(f[7], pl.src_at(7) + rp);
                NOMRT_SEAM(t[3], pl.src_at(12) + r0);
                if constexpr (TQ == 9) {
                    NOMRT_SEAM(t[6], pl.src_at(15) + rm);
                    NOMRT_SEAM(t[7], pl.src_at(16) + rp);
                }
#undef NOMRT_SEAM
            }
        }
    } else {
        // Values from beyond the warp's 128 cells, for the planes shifted along x: lane 0's
        // left neighbour (x0 - 1, wrapped on a periodic x), lane 31's right neighbour
        // (x0 + 4) and, on a periodic x, cell 0 for the lane holding cell nx - 1. One branch
        // per kind loads them for every shifted plane.
        // e_x = +1 planes (source x - 1): f1, f5, f8, t1 (+ t5, t8); e_x = -1: f3, f6, f7, t3 (+ t6, t7)
        constexpr int NE = TQ == 9 ? 6 : 4;
        const S *lrow[6] = {pl.src_at(1) + r0, pl.src_at(5) + rm, pl.src_at(8) + rp, pl.src_at(10) + r0,
                            pl.src_at(TQ == 9 ? 14 : 10) + rm, pl.src_at(TQ == 9 ? 17 : 10) + rp};
        const S *rrow[6] = {pl.src_at(3) + r0, pl.src_at(6) + rm, pl.src_at(7) + rp, pl.src_at(12) + r0,
                            pl.src_at(TQ == 9 ? 15 : 12) + rm, pl.src_at(TQ == 9 ? 16 : 12) + rp};
        int xl = x0 - 1;
        if (xl < 0 && g.px) xl += g.nx;
        const int xr = x0 + 4;
        const int kseam = g.nx - 1 - x0;
        const int seam_k = (g.px && inrow && kseam >= 0 && kseam < 4) ? kseam : -1;
        float el[NE], er[NE], es[NE];
    #pragma unroll
        for (int i = 0; i < NE; ++i) el[i] = er[i] = es[i] = 0.f;
        if (lane == 0 && inrow && xl >= 0) {
    #pragma unroll
            for (int i = 0; i < NE; ++i)
                el[i] = NOMRT_OK(g, lrow[i] + xl, sizeof(S), 17) ? Ld<S, NC>::one(lrow[i] + xl) : 0.f;
        }
        if (lane == 31 && inrow && xr < g.nx) {
    #pragma unroll
            for (int i = 0; i < NE; ++i)
                er[i] = NOMRT_OK(g, rrow[i] + xr, sizeof(S), 18) ? Ld<S, NC>::one(rrow[i] + xr) : 0.f;
        }
        if (seam_k >= 0) {
    #pragma unroll
            for (int i = 0; i < NE; ++i) es[i] = NOMRT_OK(g, rrow[i], sizeof(S), 19) ? Ld<S, NC>::one(rrow[i]) : 0.f;
        }
        float a[4];
        ld_four<S, NC>(g, pl.src_at(0) + r0, x0, inrow, f[0]);
        ld_four<S, NC>(g, pl.src_at(1) + r0, x0, inrow, a);
        pull_from_left(a, el[0], lane, f[1]);
        ld_four<S, NC>(g, pl.src_at(2) + rm, x0, inrow, f[2]);
        ld_four<S, NC>(g, pl.src_at(3) + r0, x0, inrow, a);
        pull_from_right(a, er[0], lane, seam_k, es[0], f[3]);
        ld_four<S, NC>(g, pl.src_at(4) + rp, x0, inrow, f[4]);
        ld_four<S, NC>(g, pl.src_at(5) + rm, x0, inrow, a);
        pull_from_left(a, el[1], lane, f[5]);
        ld_four<S, NC>(g, pl.src_at(6) + rm, x0, inrow, a);
        pull_from_right(a, er[1], lane, seam_k, es[1], f[6]);
        ld_four<S, NC>(g, pl.src_at(7) + rp, x0, inrow, a);
        pull_from_right(a, er[2], lane, seam_k, es[2], f[7]);
        ld_four<S, NC>(g, pl.src_at(8) + rp, x0, inrow, a);
        pull_from_left(a, el[2], lane, f[8]);
        ld_four<S, NC>(g, pl.src_at(9) + r0, x0, inrow, t[0]);
        ld_four<S, NC>(g, pl.src_at(10) + r0, x0, inrow, a);
        pull_from_left(a, el[3], lane, t[1]);
        ld_four<S, NC>(g, pl.src_at(11) + rm, x0, inrow, t[2]);
        ld_four<S, NC>(g, pl.src_at(12) + r0, x0, inrow, a);
        pull_from_right(a, er[3], lane, seam_k, es[3], t[3]);
        ld_four<S, NC>(g, pl.src_at(13) + rp, x0, inrow, t[4]);
        if constexpr (TQ == 9) {
            ld_four<S, NC>(g, pl.src_at(14) + rm, x0, inrow, a);
            pull_from_left(a, el[4], lane, t[5]);
            ld_four<S, NC>(g, pl.src_at(15) + rm, x0, inrow, a);
            pull_from_right(a, er[4], lane, seam_k, es[4], t[6]);
            ld_four<S, NC>(g, pl.src_at(16) + rp, x0, inrow, a);
            pull_from_right(a, er[5], lane, seam_k, es[5], t[7]);
            ld_four<S, NC>(g, pl.src_at(17) + rp, x0, inrow, a);
            pull_from_left(a, el[5], lane, t[8]);
        }
    }
    if (!any) return;
    if (m4 != 0u) {
        wall_links<S, 0, 4, PA, NC, TQ>(pl, g, m4, x0, r0, rm, rp, f, t);
        wall_links<S, 1, 4, PA, NC, TQ>(pl, g, m4, x0, r0, rm, rp, f, t);
        wall_links<S, 2, 4, PA, NC, TQ>(pl, g, m4, x0, r0, rm, rp, f, t);
        wall_links<S, 3, 4, PA, NC, TQ>(pl, g, m4, x0, r0, rm, rp, f, t);
    }
    collide_pair<0, 4, TQ, BGK>(r, f, t);
    collide_pair<2, 4, TQ, BGK>(r, f, t);
    if (m4 != 0u) {
        zero_solid<0, 4, TQ>(m4, f, t);
        zero_solid<1, 4, TQ>(m4, f, t);
        zero_solid<2, 4, TQ>(m4, f, t);
        zero_solid<3, 4, TQ>(m4, f, t);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i)
        if (NOMRT_OK(g, pl.dst_at(i) + r0 + x0, 4 * sizeof(S), 28)) Vec4<S>::st(pl.dst_at(i) + r0 + x0, f[i]);
#pragma unroll
    for (int i = 0; i < TQ; ++i)
        if (NOMRT_OK(g, pl.dst_at(9 + i) + r0 + x0, 4 * sizeof(S), 29)) Vec4<S>::st(pl.dst_at(9 + i) + r0 + x0, t[i]);
}

// Bulk prefetch of `bytes` bytes at p into L2 (no registers, no completion to wait for).
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%1], %0;" ::"r"(bytes), "l"(p) : "memory");
}

// Rows ahead whose segments a block of the four-cell kernel asks L2 to fetch.
// value: the population planes. FP16 storage moves half the bytes per cell, so its
// loads alone keep too few bytes in flight; FP32 needs no lead. mask: the link map,
// the first load of every warp and the one its population loads wait on (the
// early exit of solid rows depends on it), both storages. Measured on GB300 at
// 4096 x 2048, fractions of the copy peak: FP16 planes alone 16 / 64 / 160 rows
// ahead 0.928 / 0.918 / 0.824 (7 blocks/SM); planes and mask (with the dependent
// launch) 24 / 32 ahead 0.950 / 0.952 at 7 blocks/SM, 24 / 32 / 40 / 48 ahead
// 0.957 / 0.965 / 0.969 / 0.969 at 5; FP32 1.009 -> 1.013 with the mask, the
// same for a lead of 16 to 64 rows.
template <typename S>
struct PrefetchRows {
    static constexpr int value = sizeof(S) == 2 ? 48 : 0;
    static constexpr int mask = sizeof(S) == 2 ? 48 : 32;
};

// Launched as a programmatic dependent of the previous step where its grid spans
// more than one wave (launch_dependent): the block lets the next launch start its
// blocks at once, then waits until every block of the previous grid has finished
// and its writes are visible, before its first global access. Launched without
// that attribute, the wait returns at once.
template <typename S, int MINB, int TQ = 5, bool BGK = false>
__global__ void __launch_bounds__(128, MINB) k_step4(const Planes<S> pl, const Geom g, const RatesC<float> r) {
    constexpr int PF = PrefetchRows<S>::value;
    constexpr int MPF = PrefetchRows<S>::mask;
    static_assert(PF == 0 || PF == MPF, "FP16 prefetches planes and link map with one lead");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    for (int y = blockIdx.y; y < g.ny; y += gridDim.y) {
        // this block's 512-cell segment of row y + MPF: thread q < 9 + TQ asks L2 for plane q
        // (FP16 only), thread 9 + TQ (FP16) or 0 (FP32) for the link map. 16-byte aligned:
        // segments start at multiples of 512 cells, rows are pitched to 128 bytes of
        // populations, so to a multiple of 32 cells, and every region of the block starts on
        // 256 bytes
        const int t = threadIdx.x;
        if ((PF > 0 ? t <= 9 + TQ : t == 0) && y + MPF < g.ny) {
            const int xs = blockIdx.x * 512;
            const int n = min(512, g.pitch - xs);
            const size_t at = (size_t)(y + MPF) * g.pitch + xs;
            const bool map = PF == 0 || t == 9 + TQ;
            const void *pp = map ? static_cast<const void *>(g.mask + at)
                                 : static_cast<const void *>(pl.src_at(min(t, 8 + TQ)) + at);
            const unsigned bytes = map ? (unsigned)n : (unsigned)(n * sizeof(S));
            if (NOMRT_BULK_OK(g, pp, bytes, 50)) prefetch_l2_bulk(pp, bytes);
        }
        row4<S, Planes<S>, true, TQ, BGK>(pl, g, r, x0, y, lane);
    }
}

// The same step with one warp's 128-cell row segment as the unit of work instead
// of a block's 512 cells: unit u is segment u % upr of row u / upr (upr =
// ceil(pitch / 128) segments per row), four consecutive units per 128-thread
// block. Where rows are not a multiple of 512 cells, k_step4's last block of
// every row holds warps past the row's end, which keep a block slot while doing
// nothing; here only the lattice's last block can. The block asks L2 for its four
// segments of the link map (and FP16 planes) MPF rows ahead as at most two runs
// of consecutive cells (the end of one row, the start of the next; on the 64
// cavities VEC4W members ran at 0.969 of the copy peak that way against 0.947
// with a prefetch per warp). Same row code, same bits; launched like k_step4.
template <typename S, int MINB, int TQ = 5, bool BGK = false>
__global__ void __launch_bounds__(128, MINB)
    k_step4w(const Planes<S> pl, const Geom g, const RatesC<float> r, int upr, int nunits) {
    constexpr int PF = PrefetchRows<S>::value;
    constexpr int MPF = PrefetchRows<S>::mask;
    static_assert(PF == 0 || PF == MPF, "FP16 prefetches planes and link map with one lead");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31;
    const int u0 = blockIdx.x * 4;
    {
        // the block's four units as at most two runs of consecutive cells: warp 0 the first,
        // warp 1 the second (one lane per plane; FP32: the link map only, lane 0); on a
        // lattice narrower than 512 cells the units span more rows and only the first two
        // are prefetched. Each run stays within its row. 16-byte aligned: runs start at
        // multiples of 128 cells, rows are pitched to 32 cells
        const int y0 = u0 / upr, s0 = u0 - y0 * upr;
        const int n0 = min(4, upr - s0);
        const int piece = (int)(threadIdx.x >> 5);
        const int yb = y0 + piece;
        const int xb = piece == 0 ? s0 * 128 : 0;
        const int n = piece < 2 ? min((piece == 0 ? n0 : 4 - n0) * 128, g.pitch - xb) : 0;
        if (piece < 2 && n > 0 && (PF > 0 ? lane <= 9 + TQ : lane == 0) && yb + MPF < g.ny &&
            u0 + (piece == 0 ? 0 : n0) < nunits) {
            const size_t at = (size_t)(yb + MPF) * g.pitch + xb;
            const bool map = PF == 0 || lane == 9 + TQ;
            const void *pp = map ? static_cast<const void *>(g.mask + at)
                                 : static_cast<const void *>(pl.src_at(min(lane, 8 + TQ)) + at);
            const unsigned bytes = map ? (unsigned)n : (unsigned)(n * sizeof(S));
            if (NOMRT_BULK_OK(g, pp, bytes, 55)) prefetch_l2_bulk(pp, bytes);
        }
    }
    const int u = u0 + (int)(threadIdx.x >> 5);
    if (u >= nunits) return;  // the whole warp: past the lattice's last unit
    const int y = u / upr;
    const int xs = (u - y * upr) * 128;
    row4<S, Planes<S>, true, TQ, BGK>(pl, g, r, xs + 4 * lane, y, lane);
}

}  // namespace nomrt
