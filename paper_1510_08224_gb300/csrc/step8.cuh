// FP16-shifted storage: the fused step with eight cells of one row per thread.
//
// Each population plane's eight halves arrive in one 128-bit load (four half2
// words). For planes pulled from x - 1 or x + 1 (Eq. 9 / Eq. 25 with e_x = +-1)
// the words are realigned in registers with byte permutes, the element that
// crosses into the neighbouring thread's group coming from the adjacent lane
// by a word shuffle (or a direct load at a warp edge / the periodic seam).
// After realignment word k of every plane holds the pulled values of cells 2k
// and 2k+1, so a pair of cells converts with one half2 -> float2 per plane,
// collides in FP32, and packs back into the same word; the 14 words are then
// stored as 128-bit vectors. This halves the threads per cell of the
// four-cell kernel and doubles the bytes each thread keeps in flight.
#pragma once

#include "nomrt_kernels.cuh"

namespace nomrt {

__device__ __forceinline__ uint32_t half_bits(__half h) {
    uint16_t b;
    memcpy(&b, &h, 2);
    return (uint32_t)b;
}

// Realign the eight halves of one plane for the pull with x-shift DX.
// w[4]: raw words of cells x0..x0+7 (low half = even cell).
template <int DX>
__device__ __forceinline__ void realign8(const __half *row, const Geom &g, int x0, int lane, bool inrow, uint32_t w[4]) {
    if (DX == 1) {
        // cell j pulls element j - 1
        uint32_t left = __shfl_up_sync(kFull, w[3], 1);  // neighbour's element 7 in the high half
        if (lane == 0) {
            left = 0u;
            int xs = x0 - 1;
            if (xs < 0 && g.px) xs += g.nx;
            if (inrow && xs >= 0 && NOMRT_OK(g, row + xs, 2, 30)) left = half_bits(row[xs]) << 16;
        }
        const uint32_t p0 = __byte_perm(left, w[0], 0x5432);
        const uint32_t p1 = __byte_perm(w[0], w[1], 0x5432);
        const uint32_t p2 = __byte_perm(w[1], w[2], 0x5432);
        const uint32_t p3 = __byte_perm(w[2], w[3], 0x5432);
        w[0] = p0; w[1] = p1; w[2] = p2; w[3] = p3;
        if (g.px && inrow && x0 == 0 && NOMRT_OK(g, row + g.nx - 1, 2, 31))
            w[0] = (w[0] & 0xFFFF0000u) | half_bits(row[g.nx - 1]);  // periodic seam
    } else if (DX == -1) {
        // cell j pulls element j + 1
        uint32_t right = __shfl_down_sync(kFull, w[0], 1);  // neighbour's element 0 in the low half
        if (lane == 31) {
            right = 0u;
            const int xs = x0 + 8;
            if (inrow && xs < g.nx && NOMRT_OK(g, row + xs, 2, 32)) right = half_bits(row[xs]);
        }
        const uint32_t p0 = __byte_perm(w[0], w[1], 0x5432);
        const uint32_t p1 = __byte_perm(w[1], w[2], 0x5432);
        const uint32_t p2 = __byte_perm(w[2], w[3], 0x5432);
        const uint32_t p3 = __byte_perm(w[3], right, 0x5432);
        w[0] = p0; w[1] = p1; w[2] = p2; w[3] = p3;
        if (g.px && inrow) {
            const int k = g.nx - 1 - x0;  // periodic seam: x = nx - 1 pulls from x = 0
            if (k >= 0 && k < 8) {
                const uint32_t v = NOMRT_OK(g, row, 2, 33) ? half_bits(row[0]) : 0u;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (k == 2 * q) w[q] = (w[q] & 0xFFFF0000u) | v;
                    if (k == 2 * q + 1) w[q] = (w[q] & 0x0000FFFFu) | (v << 16);
                }
            }
        }
    }
}

template <int DX>
__device__ __forceinline__ void ld_plane8(const __half *row, const Geom &g, int x0, int lane, bool inrow, uint32_t w[4]) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (inrow && NOMRT_OK(g, row + x0, 16, 34)) v = __ldg(reinterpret_cast<const uint4 *>(row + x0));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    realign8<DX>(row, g, x0, lane, inrow, w);
}

// Halfway wall links of one cell with link-map byte m at column x, in place.
__device__ __forceinline__ void links8(const Planes<__half> &pl, const Geom &g, unsigned m, int x, int r0, int rm,
                                       int rp, float f[9], float t[5]) {
    if (m == 0 || m == kSolid) return;
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
            const WallDev *wd = wall_of(g, sidx[i], 35);
            if (kBoundsBuild && !wd) continue;
            f[i] = ld_at<__half>(g, pl.src[opp[i]] + r0 + x, 36) + (float)__ldg(&wd->cf[i]);
            if (i < 5)
                t[i] = (float)__ldg(&wd->tsgn) * ld_at<__half>(g, pl.src[9 + opp[i]] + r0 + x, 36) +
                       (float)__ldg(&wd->tb);
        }
    }
}

// The cell pair (2Q, 2Q+1): unpack word Q of every plane, collide, pack back.
template <int Q>
__device__ __forceinline__ void pair8(const Planes<__half> &pl, const Geom &g, const RatesC<float> &r, uint32_t mlo,
                                      uint32_t mhi, int x0, int r0, int rm, int rp, uint32_t w[kQ][4]) {
    float fa[9], ta[5], fb[9], tb[5];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        __half2 h;
        memcpy(&h, &w[i][Q], 4);
        const float2 v = __half22float2(h);
        if (i < 9) {
            fa[i] = v.x;
            fb[i] = v.y;
        } else {
            ta[i - 9] = v.x;
            tb[i - 9] = v.y;
        }
    }
    const uint32_t mword = Q < 2 ? mlo : mhi;
    const unsigned ma = (mword >> (16 * (Q & 1))) & 0xFFu;
    const unsigned mb = (mword >> (16 * (Q & 1) + 8)) & 0xFFu;
    links8(pl, g, ma, x0 + 2 * Q, r0, rm, rp, fa, ta);
    links8(pl, g, mb, x0 + 2 * Q + 1, r0, rm, rp, fb, tb);
    float2 fp[9], tp[5];
#pragma unroll
    for (int i = 0; i < 9; ++i) fp[i] = make_float2(fa[i], fb[i]);
#pragma unroll
    for (int i = 0; i < 5; ++i) tp[i] = make_float2(ta[i], tb[i]);
    collide_x<float2>(r, fp, tp);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        fa[i] = ma == kSolid ? 0.f : fp[i].x;
        fb[i] = mb == kSolid ? 0.f : fp[i].y;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ta[i] = ma == kSolid ? 0.f : tp[i].x;
        tb[i] = mb == kSolid ? 0.f : tp[i].y;
    }
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const __half2 h = i < 9 ? __floats2half2_rn(fa[i], fb[i]) : __floats2half2_rn(ta[i - 9], tb[i - 9]);
        memcpy(&w[i][Q], &h, 4);
    }
}

template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_step8h(const Planes<__half> pl, const Geom g, const RatesC<float> r) {
    const int lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 8;
    for (int y = blockIdx.y; y < g.ny; y += gridDim.y) {
        // one thread per plane asks L2 for this block's 1024-cell segment of row y + 16
        // (as the four-cell kernel does; 16-byte aligned: segments start at multiples of
        // 1024 elements, rows are 128-byte pitched)
        if (threadIdx.x < kQ && y + PrefetchRows<__half>::value < g.ny) {
            const int xs = blockIdx.x * 1024;
            const int n = min(1024, g.pitch - xs);
            const __half *pp = pl.src[threadIdx.x] + (size_t)(y + PrefetchRows<__half>::value) * g.pitch + xs;
            if (NOMRT_BULK_OK(g, pp, n * sizeof(__half), 51)) prefetch_l2_bulk(pp, (unsigned)(n * sizeof(__half)));
        }
        const int r0 = y * g.pitch;
        const bool inrow = x0 < g.pitch;
        uint2 m8 = make_uint2(0xFFFFFFFFu, 0xFFFFFFFFu);
        if (inrow && NOMRT_OK(g, g.mask + r0 + x0, 8, 37)) m8 = __ldg(reinterpret_cast<const uint2 *>(g.mask + r0 + x0));
        const bool any = (m8.x & m8.y) != 0xFFFFFFFFu;
        if (!__any_sync(kFull, any)) continue;
        int ym = y - 1, yp = y + 1;
        if (g.py) {
            ym = (ym < 0) ? ym + g.ny : ym;
            yp = (yp >= g.ny) ? yp - g.ny : yp;
        }
        // rows of a non-periodic edge hold no fluid cell, so a warp that gets here has 0 < y < ny - 1
        const int rm = ym * g.pitch, rp = yp * g.pitch;
        uint32_t w[kQ][4];
        ld_plane8<0>(pl.src[0] + r0, g, x0, lane, inrow, w[0]);
        ld_plane8<1>(pl.src[1] + r0, g, x0, lane, inrow, w[1]);
        ld_plane8<0>(pl.src[2] + rm, g, x0, lane, inrow, w[2]);
        ld_plane8<-1>(pl.src[3] + r0, g, x0, lane, inrow, w[3]);
        ld_plane8<0>(pl.src[4] + rp, g, x0, lane, inrow, w[4]);
        ld_plane8<1>(pl.src[5] + rm, g, x0, lane, inrow, w[5]);
        ld_plane8<-1>(pl.src[6] + rm, g, x0, lane, inrow, w[6]);
        ld_plane8<-1>(pl.src[7] + rp, g, x0, lane, inrow, w[7]);
        ld_plane8<1>(pl.src[8] + rp, g, x0, lane, inrow, w[8]);
        ld_plane8<0>(pl.src[9] + r0, g, x0, lane, inrow, w[9]);
        ld_plane8<1>(pl.src[10] + r0, g, x0, lane, inrow, w[10]);
        ld_plane8<0>(pl.src[11] + rm, g, x0, lane, inrow, w[11]);
        ld_plane8<-1>(pl.src[12] + r0, g, x0, lane, inrow, w[12]);
        ld_plane8<0>(pl.src[13] + rp, g, x0, lane, inrow, w[13]);
        if (!any) continue;
        pair8<0>(pl, g, r, m8.x, m8.y, x0, r0, rm, rp, w);
        pair8<1>(pl, g, r, m8.x, m8.y, x0, r0, rm, rp, w);
        pair8<2>(pl, g, r, m8.x, m8.y, x0, r0, rm, rp, w);
        pair8<3>(pl, g, r, m8.x, m8.y, x0, r0, rm, rp, w);
#pragma unroll
        for (int q = 0; q < kQ; ++q)
            if (NOMRT_OK(g, pl.dst[q] + r0 + x0, 16, 38))
                *reinterpret_cast<uint4 *>(pl.dst[q] + r0 + x0) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
}

}  // namespace nomrt
