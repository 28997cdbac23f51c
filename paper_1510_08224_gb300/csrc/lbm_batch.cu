// Batched execution of many lattices of uneven size (FP32 or FP16-shifted
// storage): every member lattice advances by one time step per launch of the
// per-step kernel, or by k steps per launch of the persistent kernel, with a
// grid barrier between its steps.
//
// Launch groups: up to kGroupLats members whose kinetic rates (s_e, s_q,
// s_eps, zeta_e, zeta_nu, varpi) agree travel in one launch. Their
// descriptors (buffers, geometry, and the eleven collision values that follow
// from each member's own nu, alpha, g beta, T0 and body force) and the
// group's shared rates form one __grid_constant__ kernel parameter. The
// shared rates sit at fixed offsets of the parameter bank, so the collision
// reads them as constant-bank operands exactly as the single-lattice kernel
// does; only the member-specific values become registers, once per row.
//
// Work: every member's rows cut into 512-cell segments (the four-cell
// kernel's 128-thread block shape): one virtual block per (member, row,
// segment), numbered member by member, row by row, with no block beyond a
// member's own width. A block of the per-step kernel finds its member by a
// binary search over the members' first virtual blocks: every value on that
// path is the same across the block (block index, parameter bank), so the
// member's descriptor stays in the per-block (uniform) registers rather than
// in each thread's (measured: a per-thread table load instead cost the FP32
// kernel 4 %). The persistent kernel's blocks draw their virtual blocks from a
// counter, so they read (member, segment, row) from a device work table. Either
// way the block runs the single-lattice row code, so a lattice stepped in a
// batch produces the same bits as when stepped alone. The per-step kernel gives each virtual block a
// block of a 1-D grid; the persistent kernel's resident blocks take runs of
// rows_per_unit consecutive virtual blocks, step after step.
//
// Ping-pong: member l reads buffer (s + flip_l) & 1 at batch step s, where
// flip_l is fixed when the lattice joins, so lattices that joined at different
// times step in lockstep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lattice_impl.h"
#include "nomrt_kernels.cuh"
#include "nomrt_lbm.h"

namespace nomrt {

constexpr int kBatchThreads = 128;
constexpr int kBatchConfigs = 5;  // resident blocks asked of ptxas: 4 + config
constexpr int kFusedConfigs = 2 * kBatchConfigs;  // FUSED: configs 5-9 are 0-4 with one row segment per warp
constexpr int kGroupLats = 64;    // members per launch (the parameter block holds their descriptors)
constexpr long long kBarrierBudgetCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kDefaultPersistentSteps = 32;

// The collision values that follow from one lattice's nu, alpha, g beta, T0
// and body force; the rest of RatesC<float> is shared by a launch group.
struct MemberRates {
    float s_nu, om_nu, h_nu, h2nu, om_a, z_a, ax, hx, Fy0, g_beta, T_ref;
};

inline MemberRates member_rates(const RatesC<float> &r) {
    return MemberRates{r.s_nu, r.om_nu, r.h_nu, r.h2nu, r.om_a, r.z_a, r.ax, r.hx, r.Fy0, r.g_beta, r.T_ref};
}

__host__ __device__ __forceinline__ void apply_member(RatesC<float> &r, const MemberRates &v) {
    r.s_nu = v.s_nu;
    r.om_nu = v.om_nu;
    r.h_nu = v.h_nu;
    r.h2nu = v.h2nu;
    r.om_a = v.om_a;
    r.z_a = v.z_a;
    r.ax = v.ax;
    r.hx = v.hx;
    r.Fy0 = v.Fy0;
    r.g_beta = v.g_beta;
    r.T_ref = v.T_ref;
}

// Whether two lattices' rates agree outside their member-specific values.
inline bool same_shared_rates(RatesC<float> a, RatesC<float> b) {
    const MemberRates z{};
    apply_member(a, z);
    apply_member(b, z);
    return std::memcmp(&a, &b, sizeof a) == 0;
}

// One member's descriptor in a launch's parameter block.
struct GridLat {
    Geom g;
    // every population plane of both buffers (buffer 0's kQ planes, then buffer 1's): read by
    // index from the parameter bank, like the single-lattice kernel's plane pointers, rather
    // than computed from a base and a stride (measured on one 4096 x 2048 member: the FP16
    // kernel 0.68 -> 0.74 of the copy peak, FP32 unchanged)
    const void *planes[2 * kQ];
    unsigned long long xb_magic;  // ceil(2^32 / xblocks): local / xblocks = (local * xb_magic) >> 32
    int flip;
    int xblocks;                  // 512-cell segments per row: ceil(pitch / 512)
    int upr;                      // 128-cell segments per row: ceil(pitch / 128)
    MemberRates v;
};

// The planes a member's step reads (buffer sel) and writes (buffer 1 - sel), from its descriptor.
template <typename S>
struct MemberPlanes {
    const GridLat &L;
    int src0, dst0;  // 0 or kQ
    __device__ __forceinline__ const S *src_at(int q) const { return static_cast<const S *>(L.planes[src0 + q]); }
    __device__ __forceinline__ S *dst_at(int q) const {
        return static_cast<S *>(const_cast<void *>(L.planes[dst0 + q]));
    }
};

struct GroupParams {
    RatesC<float> rc;           // rates shared by the group (member-specific fields overwritten per block)
    int nlats;
    int unit;                   // persistent kernel: consecutive virtual blocks per work unit
    int nvb;                    // virtual blocks per step
    const int2 *work;           // per virtual block: (member | segment << 8, row), device
    int blk0[kGroupLats + 1];   // first virtual block of each member; blk0[nlats] = nvb
    int nwb;                    // blocks of the per-warp form per step (four 128-cell units of one member each)
    int blk0w[kGroupLats + 1];  // first such block of each member; blk0w[nlats] = nwb
    GridLat lat[kGroupLats];
};
static_assert(sizeof(GroupParams) <= 32764, "a launch group's descriptors must fit the kernel parameter space");

// Row y, segment xb (cells 512 xb .. 512 xb + 511) of member `lo` of a group,
// one step at `parity`, as block (xb, y) of the single-lattice four-cell
// kernel computes it. NC: read-only loads (the per-step kernel) or
// L2-coherent ones (the persistent kernel reads what its own previous step
// wrote). The member's descriptor is read here, per row, so that nothing of it
// stays live between rows.
template <typename S, bool NC>
__device__ __forceinline__ void batch_row(const GroupParams &P, int lo, int xb, int y, int parity) {
    const GridLat &L = P.lat[lo];
    const Geom g = L.g;
    const int sel = (parity + L.flip) & 1;
    const MemberPlanes<S> pa{L, sel ? kQ : 0, sel ? 0 : kQ};
    const int xs = xb * 512;
    constexpr int PF = PrefetchRows<S>::value;
    if constexpr (PF > 0) {
        // as the single-lattice kernel: thread q < kQ asks L2 for plane q's segment PF rows
        // ahead, thread kQ for the link map's (16-byte aligned: segments start at multiples
        // of 512 cells, rows are 128-byte pitched). FP16 only: in FP32 the link-map prefetch
        // took the fused kernel from 0.92 to 0.80 of the copy peak on 64 cavities
        const int t = threadIdx.x;
        if (t <= kQ && y + PF < g.ny) {
            const int n = min(512, g.pitch - xs);
            const size_t at = (size_t)(y + PF) * g.pitch + xs;
            const void *pp = t == kQ ? static_cast<const void *>(g.mask + at)
                                     : static_cast<const void *>(pa.src_at(min(t, kQ - 1)) + at);
            const unsigned bytes = t == kQ ? (unsigned)n : (unsigned)(n * sizeof(S));
            if (NOMRT_BULK_OK(g, pp, bytes, 52)) prefetch_l2_bulk(pp, bytes);
        }
    }
    RatesC<float> r = P.rc;  // shared rates: parameter-bank operands
    apply_member(r, L.v);    // the member's own values: registers
    row4<S, MemberPlanes<S>, NC>(pa, g, r, xs + 4 * (int)threadIdx.x, y, (int)threadIdx.x & 31);
}

// Virtual block vb of a group (the per-step kernel): its member by a binary
// search over the members' first virtual blocks, then its row and segment.
template <typename S, bool NC>
__device__ __forceinline__ void batch_block_search(const GroupParams &P, int vb, int parity) {
    int lo = 0, hi = P.nlats - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.blk0[mid] <= vb) lo = mid;
        else hi = mid - 1;
    }
    const int local = vb - P.blk0[lo];
    const int y = (int)(((unsigned long long)(unsigned)local * P.lat[lo].xb_magic) >> 32);
    const int xb = local - y * P.lat[lo].xblocks;
    batch_row<S, NC>(P, lo, xb, y, parity);
}

// Virtual block vb of a group (the persistent kernel): member, segment and row
// from the work table.
template <typename S, bool NC>
__device__ __forceinline__ void batch_block_table(const GroupParams &P, int vb, int parity) {
    const int2 w = __ldg(P.work + vb);  // vb < P.nvb, the table's length (the batch's own buffer)
    batch_row<S, NC>(P, w.x & 0xFF, w.x >> 8, w.y, parity);
}

// One step of every member of a group: one block per virtual block.
template <typename S, int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB)
    k_batch_grid(const __grid_constant__ GroupParams P, int parity) {
    for (int vb = blockIdx.x; vb < P.nvb; vb += gridDim.x) batch_block_search<S, true>(P, vb, parity);
}

// Segment seg (cells 128 seg .. 128 seg + 127) of row y of member lo, one warp's
// share: the row code of batch_row on a 128-cell unit. FP16 members ask L2 for
// the segment's planes and link map PF rows ahead (one lane each); FP32 members
// go without, as in batch_row.
template <typename S, bool NC, bool WARP_PREFETCH = true>
__device__ __forceinline__ void batch_row_w(const GroupParams &P, int lo, int seg, int y, int parity, int lane) {
    const GridLat &L = P.lat[lo];
    const Geom g = L.g;
    const int sel = (parity + L.flip) & 1;
    const MemberPlanes<S> pa{L, sel ? kQ : 0, sel ? 0 : kQ};
    const int xs = seg * 128;
    constexpr int PF = PrefetchRows<S>::value;
    if constexpr (PF > 0 && WARP_PREFETCH) {
        // 16-byte aligned: xs is a multiple of 128 cells, rows are 128-byte pitched
        if (lane <= kQ && y + PF < g.ny) {
            const int n = min(128, g.pitch - xs);
            const size_t at = (size_t)(y + PF) * g.pitch + xs;
            const void *pp = lane == kQ ? static_cast<const void *>(g.mask + at)
                                        : static_cast<const void *>(pa.src_at(min(lane, kQ - 1)) + at);
            const unsigned bytes = lane == kQ ? (unsigned)n : (unsigned)(n * sizeof(S));
            if (NOMRT_BULK_OK(g, pp, bytes, 56)) prefetch_l2_bulk(pp, bytes);
        }
    }
    RatesC<float> r = P.rc;  // shared rates: parameter-bank operands
    apply_member(r, L.v);    // the member's own values: registers
    row4<S, MemberPlanes<S>, NC>(pa, g, r, xs + 4 * lane, y, lane);
}

// One step of every member of a group with one 128-cell row segment per warp:
// the FUSED kind's configs 5-9. A block takes four consecutive segments of one
// member (row by row, so they may span two rows), so rows that are not a
// multiple of 512 cells leave no warp idle but in a member's last block, while
// the member, found by a binary search over the members' first blocks, stays
// the same across the block (its descriptor in the block-uniform registers).
template <typename S, int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB)
    k_batch_grid_w(const __grid_constant__ GroupParams P, int parity) {
    const int vb = blockIdx.x;
    int lo = 0, hi = P.nlats - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.blk0w[mid] <= vb) lo = mid;
        else hi = mid - 1;
    }
    constexpr int kWarps = kBatchThreads / 32;
    const int u0 = (vb - P.blk0w[lo]) * kWarps;
    constexpr int PF = PrefetchRows<S>::value;
    if constexpr (PF > 0) {
        // FP16: the block's four segments are at most two runs of consecutive cells (the end of
        // row y0, the start of row y0 + 1); warp 0 asks L2 for the first run's planes and link
        // map PF rows ahead, warp 1 for the second's, one lane per plane (as the 512-cell
        // kernel does, in runs of up to 1 KB rather than 256-byte pieces per warp)
        const GridLat &L = P.lat[lo];
        const Geom &g = L.g;
        const int y0 = u0 / L.upr, s0 = u0 - y0 * L.upr;
        const int n0 = min(kWarps, L.upr - s0);
        const int t = (int)threadIdx.x & 31, piece = (int)threadIdx.x >> 5;
        const int y = y0 + piece;
        const int xs = piece == 0 ? s0 * 128 : 0;
        const int n = min((piece == 0 ? n0 : kWarps - n0) * 128, g.pitch - xs);
        if (piece < 2 && t <= kQ && n > 0 && y + PF < g.ny) {
            const int sel = (parity + L.flip) & 1;
            const MemberPlanes<S> pa{L, sel ? kQ : 0, sel ? 0 : kQ};
            const size_t at = (size_t)(y + PF) * g.pitch + xs;
            const void *pp = t == kQ ? static_cast<const void *>(g.mask + at)
                                     : static_cast<const void *>(pa.src_at(min(t, kQ - 1)) + at);
            const unsigned bytes = t == kQ ? (unsigned)n : (unsigned)(n * sizeof(S));
            if (NOMRT_BULK_OK(g, pp, bytes, 57)) prefetch_l2_bulk(pp, bytes);
        }
    }
    const GridLat &L = P.lat[lo];
    const int u = u0 + (int)(threadIdx.x >> 5);
    if (u >= L.g.ny * L.upr) return;  // the whole warp: past the member's last segment
    const int y = u / L.upr;
    batch_row_w<S, true, false>(P, lo, u - y * L.upr, y, parity, (int)threadIdx.x & 31);
}

template <typename S, int MINB, bool PERSISTENT>
struct GridTag {};

// Resident CTAs per SM x SMs for a kernel, computed once per device (one cache
// per kernel instantiation: TAG distinguishes kernels of the same signature).
template <typename TAG, typename K>
cudaError_t resident_grid(K kern, int *blocks) {
    static std::atomic<int> cached[kMaxDevices];  // 0: not yet computed for that device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int n = cached[dev].load(std::memory_order_acquire);
    if (n == 0) {
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, 0);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        n = (per_sm > 0 ? per_sm : 1) * sms;
        cached[dev].store(n, std::memory_order_release);
    }
    *blocks = n;
    return cudaSuccess;
}

// Grid-wide barrier of a cooperative launch. Clock-bounded: on expiry it
// records kStatusTimeout and returns false (the caller then returns).
// `expected` is the number of arrivals that completes it: the grid size (a
// larger value is the test hook lbm_batch_debug_barrier_extra).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *status, unsigned expected) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == expected) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == gen) {
                if (clock64() - t0 > kBarrierBudgetCycles) {
                    ok = 0;
                    atomicExch(status, kStatusTimeout);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// nsteps steps of every member of a group in one cooperative launch, with a
// grid barrier between steps. Within a step the resident blocks take work
// units (P.unit consecutive virtual blocks) from a step counter as they
// become free, each asking for its next unit while it works on the current
// one, so no block waits at the barrier for a neighbour that drew slower
// units. Two counters alternate between steps (ctr[s & 1]); block 0 clears
// the one just used after the barrier that ends its step, before the step
// that uses it again; the host clears both before the launch. advance = 0
// recomputes the step at parity0 nsteps times (the tuner's trials, which leave
// the state as it was). A launch that finds the status word set (an earlier
// barrier gave up: the state is undefined) returns at once.
template <typename S, int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB)
    k_batch_persistent(const __grid_constant__ GroupParams P, int parity0, int nsteps, int advance, unsigned expected,
                       unsigned *bar, unsigned *ctr, int *status) {
    if (*reinterpret_cast<volatile int *>(status) != kStatusOk) return;
    __shared__ unsigned next;
    const int U = P.unit;
    const unsigned nunits = (unsigned)((P.nvb + U - 1) / U);
    for (int s = 0; s < nsteps; ++s) {
        const int parity = parity0 + (advance ? s : 0);
        unsigned *c = ctr + (s & 1);
        if (threadIdx.x == 0) next = atomicAdd(c, 1u);
        __syncthreads();
        unsigned u = next;
        while (u < nunits) {
            __syncthreads();  // every thread has read `next`
            if (threadIdx.x == 0) next = atomicAdd(c, 1u);
            const int v0 = (int)u * U, v1 = min(v0 + U, P.nvb);
            for (int vb = v0; vb < v1; ++vb) batch_block_table<S, false>(P, vb, parity);
            __syncthreads();
            u = next;
        }
        if (s + 1 < nsteps) {
            if (!grid_barrier(bar, status, expected)) return;
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(c, 0u);  // ready for step s + 2
        }
    }
}

template <typename S, int MINB>
cudaError_t launch_grid_shape(const GroupParams &G, int parity, cudaStream_t st) {
    if (G.nvb == 0) return cudaSuccess;
    k_batch_grid<S, MINB><<<G.nvb, kBatchThreads, 0, st>>>(G, parity);
    return cudaGetLastError();
}

template <typename S, int MINB>
cudaError_t launch_grid_w_shape(const GroupParams &G, int parity, cudaStream_t st) {
    if (G.nwb == 0) return cudaSuccess;
    k_batch_grid_w<S, MINB><<<G.nwb, kBatchThreads, 0, st>>>(G, parity);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_batch_grid(int config, const GroupParams &G, int parity, cudaStream_t st) {
    switch (config) {
        case 5: return launch_grid_w_shape<S, 4>(G, parity, st);
        case 6: return launch_grid_w_shape<S, 5>(G, parity, st);
        case 7: return launch_grid_w_shape<S, 6>(G, parity, st);
        case 8: return launch_grid_w_shape<S, 7>(G, parity, st);
        case 9: return launch_grid_w_shape<S, 8>(G, parity, st);
        case 1: return launch_grid_shape<S, 5>(G, parity, st);
        case 2: return launch_grid_shape<S, 6>(G, parity, st);
        case 3: return launch_grid_shape<S, 7>(G, parity, st);
        case 4: return launch_grid_shape<S, 8>(G, parity, st);
        default: return launch_grid_shape<S, 4>(G, parity, st);
    }
}

template <typename S, int MINB>
cudaError_t launch_persistent_shape(const GroupParams &G, int parity, int nsteps, int advance, int barrier_extra,
                                    unsigned *bar, unsigned *ctr, int *status, cudaStream_t st) {
    if (G.nvb == 0 || nsteps <= 0) return cudaSuccess;
    auto kern = k_batch_persistent<S, MINB>;
    int blocks = 0;
    cudaError_t e = resident_grid<GridTag<S, MINB, true>>(kern, &blocks);
    if (e != cudaSuccess) return e;
    const int units = (G.nvb + G.unit - 1) / G.unit;
    if (blocks > units) blocks = units;  // every block finds a first unit
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const unsigned expected = (unsigned)(blocks + barrier_extra);
    e = cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, kern, G, parity, nsteps, advance, expected, bar, ctr, status);
}

template <typename S>
cudaError_t launch_batch_persistent(int config, const GroupParams &G, int parity, int nsteps, int advance,
                                    int barrier_extra, unsigned *bar, int *status, cudaStream_t st) {
    unsigned *ctr = bar + 2;  // the two step counters follow the barrier's words
    switch (config % kBatchConfigs) {  // the per-warp configs of the FUSED kind map to their occupancy
        case 1: return launch_persistent_shape<S, 5>(G, parity, nsteps, advance, barrier_extra, bar, ctr, status, st);
        case 2: return launch_persistent_shape<S, 6>(G, parity, nsteps, advance, barrier_extra, bar, ctr, status, st);
        case 3: return launch_persistent_shape<S, 7>(G, parity, nsteps, advance, barrier_extra, bar, ctr, status, st);
        case 4: return launch_persistent_shape<S, 8>(G, parity, nsteps, advance, barrier_extra, bar, ctr, status, st);
        default: return launch_persistent_shape<S, 4>(G, parity, nsteps, advance, barrier_extra, bar, ctr, status, st);
    }
}

}  // namespace nomrt

struct lbm_batch {
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only for graph capture
    int storage = -1;
    std::vector<lbm_lattice *> members;
    std::vector<int> flip;
    int64_t s = 0;  // batch steps taken
    // device words of the persistent kernel (allocated by the batch)
    unsigned *d_bar = nullptr;
    int *d_status = nullptr;
    // the launch groups' work tables (int2 per virtual block, groups side by side)
    int2 *d_work = nullptr;
    size_t cap_work = 0;
    // lbm_batch_residuals: the members' five residual sums on the device and their pinned host copy
    double *d_res = nullptr;
    double *h_res = nullptr;
    size_t cap_res = 0;
    std::vector<nomrt::GroupParams> groups;  // launch parameters, kGroupLats members each
    int64_t cells = 0;
    int nunits = 0;  // (row chunk, segment) virtual blocks per step
    bool dirty = true;
    int config = -1;  // -1: default per storage
    int steps_per_launch = nomrt::kDefaultPersistentSteps;
    int graph_steps = 32;
    int rows_per_unit = 1;
    int barrier_extra = 0;  // test hook: grid-barrier arrivals that never come
    int kind = LBM_BATCH_FUSED;
    // concurrent kind: the step kernel every member runs (LBM_STEP_AUTO: each member's own choice)
    int member_variant = LBM_STEP_AUTO;
    int member_config = 0;
    // concurrent kind: one stream per member for the fork/join of the graph
    std::vector<cudaStream_t> lstreams;
    std::vector<cudaEvent_t> levents;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t graph = nullptr;
    // the members' step kernels (variant, config) when the graph was captured: a concurrent
    // batch's graph holds them, so a member's later lbm_set_step_kernel drops the graph
    std::vector<int2> graph_kernels;
    std::string err;

    // the default: FP32 one 128-cell row segment per warp at 5 blocks/SM (64 cavities 0.962 of the
    // copy peak against 0.924 for one 512-cell segment per block; serving 32-128-cell lattices
    // 22.7 against 18.3 solves/s), FP16 one 512-cell segment per block at 7 blocks/SM
    int cfg() const { return config >= 0 ? config : (storage == LBM_F16_SHIFTED ? 3 : 6); }
};

namespace {

lbm_status bfail(lbm_batch *b, lbm_status st, const std::string &m) {
    if (b) b->err = m;
    else nomrt::set_thread_error(m.c_str());
    return st;
}

lbm_status bcuda(lbm_batch *b, cudaError_t e, const char *what) {
    return bfail(b, LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void drop_graph(lbm_batch *b) {
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

// Rebuild the launch groups after a membership or shape change: members join
// the first group whose shared rates equal theirs and that has room.
lbm_status rebuild(lbm_batch *b) {
    if (!b->dirty) return LBM_OK;
    drop_graph(b);
    b->cells = 0;
    b->groups.clear();
    for (size_t l = 0; l < b->members.size(); ++l) {
        lbm_lattice *h = b->members[l];
        const nomrt::KParams &kp = h->kp;
        const nomrt::RatesC<float> r = nomrt::make_rates<float>(kp);
        b->cells += h->fluid;
        nomrt::GroupParams *G = nullptr;
        for (nomrt::GroupParams &c : b->groups)
            if (c.nlats < nomrt::kGroupLats && nomrt::same_shared_rates(c.rc, r)) {
                G = &c;
                break;
            }
        if (!G) {
            b->groups.emplace_back();
            G = &b->groups.back();
            std::memset(G, 0, sizeof(nomrt::GroupParams));
            G->rc = r;
        }
        nomrt::GridLat &gl = G->lat[G->nlats];
        gl.g = nomrt::make_geom(kp);
        const size_t eb = h->storage == LBM_F16_SHIFTED ? 2 : 4;
        for (int buf = 0; buf < 2; ++buf)
            for (int q = 0; q < nomrt::kQ; ++q)
                gl.planes[buf * nomrt::kQ + q] = static_cast<const char *>(kp.pop[buf]) + (size_t)q * kp.plane * eb;
        gl.flip = b->flip[l];
        gl.xblocks = (kp.pitch / 4 + nomrt::kBatchThreads - 1) / nomrt::kBatchThreads;
        gl.xb_magic = ((1ULL << 32) + (unsigned long long)gl.xblocks - 1) / (unsigned long long)gl.xblocks;
        gl.v = nomrt::member_rates(r);
        gl.upr = (kp.pitch + 127) / 128;
        G->blk0w[G->nlats + 1] = G->blk0w[G->nlats] + (kp.ny * gl.upr + nomrt::kBatchThreads / 32 - 1) /
                                                         (nomrt::kBatchThreads / 32);
        G->nwb = G->blk0w[G->nlats + 1];
        G->unit = b->rows_per_unit;
        G->blk0[G->nlats + 1] = G->blk0[G->nlats] + kp.ny * gl.xblocks;
        G->nvb = G->blk0[G->nlats + 1];
        G->nlats += 1;
    }
    // work tables: each group's virtual blocks member by member, row by row, segment by segment
    size_t total = 0;
    for (const nomrt::GroupParams &G : b->groups) total += (size_t)G.nvb;
    std::vector<int2> work(total);
    size_t at = 0;
    for (const nomrt::GroupParams &G : b->groups)
        for (int m = 0; m < G.nlats; ++m)
            for (int y = 0; y < G.lat[m].g.ny; ++y)
                for (int xb = 0; xb < G.lat[m].xblocks; ++xb) work[at++] = make_int2(m | (xb << 8), y);
    if (total > b->cap_work) {
        cudaError_t e = cudaStreamSynchronize(b->stream);  // the old table may still be in use
        if (b->d_work) cudaFree(b->d_work);
        b->d_work = nullptr;
        b->cap_work = 0;
        const size_t want = std::max<size_t>(total * 5 / 4, 1024);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_work, want * sizeof(int2));
        if (e != cudaSuccess) return bcuda(b, e, "batch work table");
        b->cap_work = want;
    }
    if (total) {
        // the host vector goes away after this call: copy and wait
        cudaError_t e = cudaMemcpyAsync(b->d_work, work.data(), total * sizeof(int2), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "upload work table");
    }
    b->nunits = 0;
    at = 0;
    for (nomrt::GroupParams &G : b->groups) {
        G.work = b->d_work + at;
        at += (size_t)G.nvb;
        b->nunits += G.nvb;
    }
    b->dirty = false;
    return LBM_OK;
}

cudaError_t ensure_streams(lbm_batch *b) {
    cudaError_t e = cudaSuccess;
    if (!b->fork) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    while (e == cudaSuccess && b->lstreams.size() < b->members.size()) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            b->lstreams.push_back(s);
            b->levents.push_back(ev);
        }
    }
    return e;
}

// n steps of every member with each member's own step kernel (its AUTO or
// chosen variant), each member on its own stream between a fork and a join on
// `st`, so the members' kernels can run concurrently. advance = false re-runs
// the current step n times without advancing (tuning).
// The parameters a member's step runs with in the concurrent kind: its own, with the
// batch's member kernel in place of its own choice where one is set.
nomrt::KParams member_params(const lbm_batch *b, const lbm_lattice *h) {
    nomrt::KParams q = h->kp;
    if (b->member_variant != LBM_STEP_AUTO) {
        q.variant = b->member_variant;
        q.config = b->member_config;
    }
    return q;
}

cudaError_t launch_concurrent(lbm_batch *b, int n, cudaStream_t st, bool advance) {
    cudaError_t e = ensure_streams(b);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(b->fork, st);
    if (e != cudaSuccess) return e;
    // largest members first, so the small ones fill in around them
    std::vector<size_t> order(b->members.size());
    for (size_t l = 0; l < order.size(); ++l) order[l] = l;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t c) { return b->members[a]->fluid > b->members[c]->fluid; });
    for (size_t l : order) {
        lbm_lattice *h = b->members[l];
        cudaStream_t ls = b->lstreams[l];
        e = cudaStreamWaitEvent(ls, b->fork, 0);
        if (e != cudaSuccess) return e;
        int cur = h->cur;
        const nomrt::KParams q = member_params(b, h);
        for (int k = 0; k < n; ++k) {
            e = h->L->step(q, cur, ls);
            if (e != cudaSuccess) return e;
            if (advance) cur ^= 1;
        }
        e = cudaEventRecord(b->levents[l], ls);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->levents[l], 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The boundary nodes of NEE walls of every member, for the batch step at
// `parity` (after the fused kernel, which skips them).
cudaError_t launch_nee_passes(lbm_batch *b, int parity, cudaStream_t st) {
    for (size_t l = 0; l < b->members.size(); ++l) {
        lbm_lattice *h = b->members[l];
        if (h->kp.n_nee == 0) continue;
        cudaError_t e = h->L->nee(h->kp, (parity + b->flip[l]) & 1, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool any_nee(const lbm_batch *b) {
    for (const lbm_lattice *h : b->members)
        if (h->kp.n_nee > 0) return true;
    return false;
}

// One step of every member with the per-step fused kernel: one launch per group.
cudaError_t launch_grid_step(lbm_batch *b, int config, int parity, cudaStream_t st) {
    for (const nomrt::GroupParams &G : b->groups) {
        cudaError_t e = b->storage == LBM_F16_SHIFTED ? nomrt::launch_batch_grid<__half>(config, G, parity, st)
                                                      : nomrt::launch_batch_grid<float>(config, G, parity, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// k steps of every member with the persistent kernel: one launch per group
// (groups hold disjoint lattices, so they need no barrier between them).
cudaError_t launch_persistent_steps(lbm_batch *b, int config, int parity, int k, int advance, cudaStream_t st) {
    for (const nomrt::GroupParams &G : b->groups) {
        cudaError_t e = b->storage == LBM_F16_SHIFTED
                            ? nomrt::launch_batch_persistent<__half>(config, G, parity, k, advance, b->barrier_extra,
                                                                     b->d_bar, b->d_status, st)
                            : nomrt::launch_batch_persistent<float>(config, G, parity, k, advance, b->barrier_extra,
                                                                    b->d_bar, b->d_status, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_steps(lbm_batch *b, int parity, int n, cudaStream_t st) {
    if (b->kind == LBM_BATCH_CONCURRENT) return launch_concurrent(b, n, st, true);
    // members with NEE walls need their boundary-node pass between steps: one launch per step
    if (b->kind == LBM_BATCH_PERSISTENT && !any_nee(b)) {
        while (n > 0) {
            const int k = std::min(n, b->steps_per_launch);
            cudaError_t e = launch_persistent_steps(b, b->cfg(), parity, k, 1, st);
            if (e != cudaSuccess) return e;
            parity = (parity + k) & 1;
            n -= k;
        }
        return cudaSuccess;
    }
    const bool nee = any_nee(b);
    for (; n > 0; --n) {
        cudaError_t e = launch_grid_step(b, b->cfg(), parity, st);
        if (e == cudaSuccess && nee) e = launch_nee_passes(b, parity, st);
        if (e != cudaSuccess) return e;
        parity ^= 1;
    }
    return cudaSuccess;
}

std::vector<int2> member_kernels(const lbm_batch *b) {
    std::vector<int2> k;
    k.reserve(b->members.size());
    for (const lbm_lattice *h : b->members) {
        const nomrt::KParams q = member_params(b, h);
        k.push_back(make_int2(q.variant, q.config));
    }
    return k;
}

bool same_kernels(const std::vector<int2> &a, const std::vector<int2> &c) {
    if (a.size() != c.size()) return false;
    for (size_t i = 0; i < a.size(); ++i)
        if (a[i].x != c[i].x || a[i].y != c[i].y) return false;
    return true;
}

lbm_status ensure_graph(lbm_batch *b) {
    if (b->graph && b->kind == LBM_BATCH_CONCURRENT && !same_kernels(b->graph_kernels, member_kernels(b)))
        drop_graph(b);
    if (b->graph || b->graph_steps <= 0) return LBM_OK;
    b->graph_kernels = member_kernels(b);
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "begin capture");
    cudaError_t le = launch_steps(b, 0, b->graph_steps, b->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, le != cudaSuccess ? le : e, "graph capture");
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bcuda(b, e, "graph instantiate");
    }
    return LBM_OK;
}

}  // namespace

// Called by lbm_destroy for a lattice still in a batch.
void nomrt::batch_detach(lbm_batch *b, lbm_lattice *h) { lbm_batch_remove(b, h); }

extern "C" {

lbm_status lbm_batch_create(void *cuda_stream, lbm_batch **out) {
    if (!out) return bfail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ENOMEM, "host allocation failed");
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_bar, 4 * sizeof(unsigned));  // barrier (count, generation), 2 step counters
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_bar, 0, 4 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        lbm_status st = bcuda(nullptr, e, "batch set-up");
        lbm_batch_destroy(b);
        return st;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_add(lbm_batch *b, lbm_lattice *h) {
    if (!b || !h) return bfail(b, LBM_EINVAL, "batch or lattice is NULL");
    if (h->batch) return bfail(b, LBM_EINVAL, "lattice already belongs to a batch");
    if (h->storage == LBM_F64) return bfail(b, LBM_EINVAL, "batches hold FP32 or FP16 storage only");
    if (h->kp.tq != 5 || h->kp.bgk)
        return bfail(b, LBM_EINVAL, "batches hold MRT lattices with the D2Q5 temperature model only");
    if (b->storage >= 0 && h->storage != b->storage) return bfail(b, LBM_EINVAL, "batch members share one storage");
    if (h->stream != b->stream) return bfail(b, LBM_EINVAL, "a member must use the batch's stream");
    b->storage = h->storage;
    b->members.push_back(h);
    b->flip.push_back((int)((h->cur + b->s) & 1));
    h->batch = b;
    b->dirty = true;
    return LBM_OK;
}

lbm_status lbm_batch_remove(lbm_batch *b, lbm_lattice *h) {
    if (!b || !h) return bfail(b, LBM_EINVAL, "batch or lattice is NULL");
    auto it = std::find(b->members.begin(), b->members.end(), h);
    if (it == b->members.end()) return bfail(b, LBM_EINVAL, "lattice is not in this batch");
    const size_t i = (size_t)(it - b->members.begin());
    b->members.erase(it);
    b->flip.erase(b->flip.begin() + (long)i);
    h->batch = nullptr;
    if (b->members.empty()) b->storage = -1;
    b->dirty = true;
    return LBM_OK;
}

lbm_status lbm_batch_set_mode(lbm_batch *b, int32_t steps_per_launch, int32_t graph_steps) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (steps_per_launch < 1) return bfail(b, LBM_EINVAL, "steps_per_launch must be >= 1");
    if (graph_steps < 0 || (graph_steps % 2) != 0) return bfail(b, LBM_EINVAL, "graph_steps must be even and >= 0");
    b->steps_per_launch = steps_per_launch;
    b->graph_steps = graph_steps;
    drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_set_kind(lbm_batch *b, int32_t kind) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (kind != LBM_BATCH_FUSED && kind != LBM_BATCH_CONCURRENT && kind != LBM_BATCH_PERSISTENT)
        return bfail(b, LBM_EINVAL, "unknown batch kind");
    b->kind = kind;
    drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_set_config(lbm_batch *b, int32_t config, int32_t rows_per_unit) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (config < -1 || config >= nomrt::kFusedConfigs) return bfail(b, LBM_EINVAL, "config out of range");
    if (rows_per_unit < 1 || rows_per_unit > 1024) return bfail(b, LBM_EINVAL, "rows_per_unit must be 1..1024");
    b->config = config;
    if (rows_per_unit != b->rows_per_unit) {
        b->rows_per_unit = rows_per_unit;
        b->dirty = true;
    }
    drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_set_member_kernel(lbm_batch *b, int32_t variant, int32_t config) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    const bool ok = (variant == LBM_STEP_AUTO && config == 0) || (variant == LBM_STEP_SCALAR && config == 0) ||
                    ((variant == LBM_STEP_VEC4 || variant == LBM_STEP_VEC4W) && config >= 0 && config < 5);
    if (!ok) return bfail(b, LBM_EINVAL, "member kernel must be AUTO, SCALAR, or VEC4 / VEC4W with config 0..4");
    b->member_variant = variant;
    b->member_config = config;
    drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_get_member_kernel(const lbm_batch *b, int32_t *variant, int32_t *config) {
    if (!b) return LBM_EINVAL;
    if (variant) *variant = b->member_variant;
    if (config) *config = b->member_config;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (nsteps < 0) return bfail(b, LBM_EINVAL, "nsteps must be >= 0");
    if (b->members.empty() || nsteps == 0) return LBM_OK;
    lbm_status st = rebuild(b);
    if (st != LBM_OK) return st;
    int64_t left = nsteps;
    auto advance = [&](int64_t k) {
        b->s += k;
        left -= k;
        for (lbm_lattice *h : b->members) {
            h->cur = (int)((h->cur + k) & 1);
            h->steps += k;
        }
    };
    while (left > 0) {
        const int parity = (int)(b->s & 1);
        if (b->graph_steps > 0 && parity == 0 && left >= b->graph_steps) {
            st = ensure_graph(b);
            if (st != LBM_OK) return st;
            cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "graph launch");
            advance(b->graph_steps);
            continue;
        }
        // direct launches: one step to reach even parity, or the remainder
        int64_t k = (b->graph_steps > 0 && parity == 1) ? 1 : left;
        k = std::min<int64_t>(k, 1 << 20);
        cudaError_t e = launch_steps(b, parity, (int)k, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "batch step launch");
        advance(k);
    }
    return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch *b) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch sync");
    int st = 0;
    e = cudaMemcpy(&st, b->d_status, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "read batch status");
    if (st != nomrt::kStatusOk) {
        const int zero = 0;
        cudaMemcpy(b->d_status, &zero, sizeof zero, cudaMemcpyHostToDevice);
        cudaMemset(b->d_bar, 0, 4 * sizeof(unsigned));
        return bfail(b, LBM_ETIMEOUT, "the persistent batch kernel gave up a grid barrier");
    }
    if constexpr (nomrt::kBoundsBuild) {
        // the members' bounds words (the word after each lattice's status word)
        for (lbm_lattice *h : b->members) {
            int w = 0;
            e = cudaMemcpy(&w, h->kp.oob, sizeof w, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return bcuda(b, e, "read bounds word");
            if (w != 0) {
                const int zero = 0;
                cudaMemcpy(h->kp.oob, &zero, sizeof zero, cudaMemcpyHostToDevice);
                return bfail(b, LBM_ECUDA,
                             "bounds-checking build: an index check failed at site " + std::to_string(w) +
                                 " in a batch member (the access was skipped; the state is invalid)");
            }
        }
    }
    return LBM_OK;
}

lbm_status lbm_batch_debug_barrier_extra(lbm_batch *b, int32_t extra) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (extra < 0 || extra > 1) return bfail(b, LBM_EINVAL, "extra must be 0 or 1");
    b->barrier_extra = extra;
    drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch *b, int32_t trial_steps, int32_t *best_kind, int32_t *best_config,
                          float *ms_per_step) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (trial_steps < 2) return bfail(b, LBM_EINVAL, "trial_steps must be >= 2");
    if (b->members.empty()) return bfail(b, LBM_EINVAL, "batch is empty");
    // Every trial re-runs the current step with the same source parity: it
    // rewrites the destination buffers with the same values and leaves the
    // state the next real step reads untouched.
    const int parity = (int)(b->s & 1);
    const bool nee = any_nee(b);
    const int k = b->steps_per_launch > 1 ? b->steps_per_launch : nomrt::kDefaultPersistentSteps;
    // candidates: FUSED configs 0-9, PERSISTENT configs 0-4 with work units of one and of two row
    // segments, CONCURRENT with the members' own kernels, then CONCURRENT with every member on
    // VEC4 and on VEC4W at each config
    constexpr int kPers = nomrt::kFusedConfigs;
    constexpr int kPersUnits = 2;
    constexpr int kConc = kPers + kPersUnits * nomrt::kBatchConfigs;
    constexpr int kCand = kConc + 1 + 2 * nomrt::kBatchConfigs;
    float ms[kCand];
    for (float &m : ms) m = INFINITY;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, LBM_ECUDA, "event create");
    lbm_status out = rebuild(b);
    // time `run(n)` for n = trial_steps after one warm-up call of run(1 or k)
    auto timed = [&](auto run, int warm, float *dst) -> cudaError_t {
        cudaError_t e = run(warm);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = run(trial_steps);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess) *dst = t / (float)trial_steps;
        return e;
    };
    for (int c = 0; c < nomrt::kFusedConfigs && out == LBM_OK; ++c) {
        cudaError_t e = timed(
            [&](int n) -> cudaError_t {
                for (int i = 0; i < n; ++i) {
                    cudaError_t le = launch_grid_step(b, c, parity, b->stream);
                    if (le == cudaSuccess && nee) le = launch_nee_passes(b, parity, b->stream);
                    if (le != cudaSuccess) return le;
                }
                return cudaSuccess;
            },
            1, &ms[c]);
        if (e != cudaSuccess) out = bcuda(b, e, "tuning launch (fused)");
    }
    // the work unit is a launch parameter only (the work table does not depend on it)
    auto set_unit = [&](int u) {
        for (nomrt::GroupParams &G : b->groups) G.unit = u;
    };
    for (int pu = 0; pu < kPersUnits && out == LBM_OK && !nee; ++pu) {
        set_unit(pu + 1);
        for (int c = 0; c < nomrt::kBatchConfigs && out == LBM_OK; ++c) {
            cudaError_t e = timed(
                [&](int n) -> cudaError_t {
                    for (int done = 0; done < n;) {
                        const int m = std::min(k, n - done);
                        cudaError_t le = launch_persistent_steps(b, c, parity, m, 0, b->stream);
                        if (le != cudaSuccess) return le;
                        done += m;
                    }
                    return cudaSuccess;
                },
                std::min(k, trial_steps), &ms[kPers + pu * nomrt::kBatchConfigs + c]);
            if (e != cudaSuccess) out = bcuda(b, e, "tuning launch (persistent)");
        }
    }
    set_unit(b->rows_per_unit);
    const int own_variant = b->member_variant, own_config = b->member_config;
    for (int c = 0; c <= 2 * nomrt::kBatchConfigs && out == LBM_OK; ++c) {
        b->member_variant = c == 0 ? LBM_STEP_AUTO : c <= nomrt::kBatchConfigs ? LBM_STEP_VEC4 : LBM_STEP_VEC4W;
        b->member_config = c == 0 ? 0 : (c - 1) % nomrt::kBatchConfigs;
        cudaError_t e = timed([&](int n) { return launch_concurrent(b, n, b->stream, false); }, 1, &ms[kConc + c]);
        if (e != cudaSuccess) out = bcuda(b, e, "tuning launch (concurrent)");
    }
    b->member_variant = own_variant;
    b->member_config = own_config;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (out != LBM_OK) return out;
    // a barrier that gave up during a trial is reported by the next lbm_batch_sync
    int best = 0;
    for (int c = 1; c < kCand; ++c)
        if (ms[c] < ms[best]) best = c;
    if (best < kPers) {
        b->kind = LBM_BATCH_FUSED;
        b->config = best;
    } else if (best < kConc) {
        b->kind = LBM_BATCH_PERSISTENT;
        b->config = (best - kPers) % nomrt::kBatchConfigs;
        b->rows_per_unit = (best - kPers) / nomrt::kBatchConfigs + 1;
        set_unit(b->rows_per_unit);
        b->steps_per_launch = k;
    } else {
        b->kind = LBM_BATCH_CONCURRENT;
        const int c = best - kConc;
        b->member_variant = c == 0 ? LBM_STEP_AUTO : c <= nomrt::kBatchConfigs ? LBM_STEP_VEC4 : LBM_STEP_VEC4W;
        b->member_config = c == 0 ? 0 : (c - 1) % nomrt::kBatchConfigs;
    }
    drop_graph(b);
    if (best_kind) *best_kind = b->kind;
    if (best_config) *best_config = b->kind == LBM_BATCH_CONCURRENT ? best - kConc - 1 : b->config;
    if (ms_per_step)
        for (int c = 0; c < kCand; ++c) ms_per_step[c] = ms[c];
    return LBM_OK;
}

lbm_status lbm_batch_info(const lbm_batch *b, int32_t *members, int64_t *cells, int32_t *units, int32_t *config,
                          int32_t *rows_per_unit, int64_t *steps_done) {
    if (!b) return LBM_EINVAL;
    if (members) *members = (int32_t)b->members.size();
    if (cells) {
        int64_t c = 0;
        for (const lbm_lattice *h : b->members) c += h->fluid;
        *cells = c;
    }
    if (units) *units = b->nunits;
    if (config) *config = b->kind == LBM_BATCH_CONCURRENT ? -1 : b->cfg();
    if (rows_per_unit) *rows_per_unit = b->rows_per_unit;
    if (steps_done) *steps_done = b->s;
    return LBM_OK;
}

lbm_status lbm_batch_residuals(lbm_batch *b, int32_t cap, lbm_lattice **members, double *r, int32_t *n) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    const int m = (int)b->members.size();
    if (n) *n = m;
    if (cap < m) return bfail(b, LBM_EINVAL, "cap is smaller than the number of members");
    if (m == 0) return LBM_OK;
    if (!r) return bfail(b, LBM_EINVAL, "r is NULL");
    if ((size_t)m > b->cap_res) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (b->d_res) cudaFree(b->d_res);
        if (b->h_res) cudaFreeHost(b->h_res);
        b->d_res = nullptr;
        b->h_res = nullptr;
        b->cap_res = 0;
        const size_t want = std::max<size_t>((size_t)m * 3 / 2, 64);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_res, want * 5 * sizeof(double));
        if (e == cudaSuccess) e = cudaHostAlloc(&b->h_res, want * 5 * sizeof(double), cudaHostAllocDefault);
        if (e != cudaSuccess) return bcuda(b, e, "residual buffers");
        b->cap_res = want;
    }
    // every member's residual kernels on the batch's stream, their sums side by side
    for (int i = 0; i < m; ++i) {
        lbm_lattice *h = b->members[i];
        cudaError_t e = h->L->residual(h->kp, h->cur, h->snap(), h->have_snap, h->partials(), b->stream);
        if (e == cudaSuccess) e = nomrt::reduce_partials(h->partials(), 5, b->d_res + 5 * (size_t)i, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "residual kernels");
    }
    cudaError_t e = cudaMemcpyAsync(b->h_res, b->d_res, (size_t)m * 5 * sizeof(double), cudaMemcpyDeviceToHost,
                                    b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "read residuals");
    lbm_status st = lbm_batch_sync(b);
    if (st != LBM_OK) return st;
    for (int i = 0; i < m; ++i) {
        lbm_lattice *h = b->members[i];
        const double *q = b->h_res + 5 * (size_t)i;
        if (members) members[i] = h;
        const int had = h->have_snap;
        h->have_snap = 1;
        if (q[4] > 0.0 || !std::isfinite(q[0]) || !std::isfinite(q[1]) || !std::isfinite(q[2]) ||
            !std::isfinite(q[3])) {
            r[i] = NAN;
        } else if (!had) {
            r[i] = INFINITY;
        } else {
            const double Ru = std::sqrt(q[0]) / std::max(std::sqrt(q[1]), 1e-300);
            const double RT = std::sqrt(q[2]) / std::max(std::sqrt(q[3]), 1e-300);
            r[i] = std::max(Ru, RT);
        }
    }
    return LBM_OK;
}

lbm_status lbm_batch_get_mode(const lbm_batch *b, int32_t *kind, int32_t *steps_per_launch, int32_t *graph_steps) {
    if (!b) return LBM_EINVAL;
    if (kind) *kind = b->kind;
    if (steps_per_launch) *steps_per_launch = b->steps_per_launch;
    if (graph_steps) *graph_steps = b->graph_steps;
    return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) {
    if (!b) return lbm_last_error(nullptr);
    return b->err.c_str();
}

void lbm_batch_destroy(lbm_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (lbm_lattice *h : b->members) h->batch = nullptr;
    drop_graph(b);
    for (cudaStream_t ls : b->lstreams) cudaStreamDestroy(ls);
    for (cudaEvent_t ev : b->levents) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->d_bar) cudaFree(b->d_bar);
    if (b->d_status) cudaFree(b->d_status);
    if (b->d_res) cudaFree(b->d_res);
    if (b->h_res) cudaFreeHost(b->h_res);
    if (b->d_work) cudaFree(b->d_work);
    delete b;
}

}  // extern "C"
