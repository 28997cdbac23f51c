// Batched execution of many lattices of uneven size (FP32 or FP16-shifted
// storage): one kernel launch advances every member lattice by one time step
// (or, in persistent mode, by k steps with a grid barrier between them).
//
// Per-step launch: the descriptors of up to kGroupLats members (buffers,
// geometry, rates) travel as one large kernel parameter, so they sit in the
// constant bank exactly as a single-lattice kernel's parameters do. The grid
// is the concatenation of every member's own VEC4 grid (one 128-thread block
// per 512-cell segment of a row); a block finds its member by a binary search
// over the members' first block indices and runs the single-lattice row code,
// so a lattice stepped in a batch produces the same bits as when stepped alone,
// and the members' partial last waves fill each other.
//
// Persistent launch: a work list of units (lattice, first row, 128-cell
// segment, row count) with the descriptors in device memory; a grid of
// resident CTAs strides over the units, steps separated by a grid barrier.
//
// Ping-pong: member l reads buffer (s + flip_l) & 1 at batch step s, where
// flip_l is fixed when the lattice joins, so lattices that joined at different
// times step in lockstep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lattice_impl.h"
#include "nomrt_kernels.cuh"
#include "nomrt_lbm.h"

namespace nomrt {

constexpr int kBatchWarps = 4;  // warps (units) per CTA
constexpr int kBatchThreads = 32 * kBatchWarps;
constexpr int kBatchConfigs = 5;  // resident blocks asked of ptxas: 4 + config
constexpr int kGroupLats = 64;    // members per per-step launch (parameter space holds their descriptors)
constexpr long long kBarrierBudgetCycles = 4000000000LL;  // ~2 s at 2 GHz

struct __align__(16) BatchLat {
    const void *pop0;
    const void *pop1;
    long long plane;
    const uint8_t *mask;
    const uint8_t *flags;
    const WallDev *walls;
    int nx, ny, pitch, px, py, flip;
    RatesC<float> r;
};

template <typename S, bool NC>
__device__ __forceinline__ void batch_unit(const BatchLat *lats, const int4 u, int parity, int lane) {
    // u = (lattice, first row, segment start, rows)
    const BatchLat *L = lats + u.x;
    Geom g;
    g.nx = L->nx;
    g.ny = L->ny;
    g.pitch = L->pitch;
    g.px = L->px;
    g.py = L->py;
    g.mask = L->mask;
    g.flags = L->flags;
    g.walls = L->walls;
    const int sel = (parity + L->flip) & 1;
    StridedPlanes<S> pa;
    pa.src = static_cast<const S *>(sel ? L->pop1 : L->pop0);
    pa.dst = static_cast<S *>(const_cast<void *>(sel ? L->pop0 : L->pop1));
    pa.plane = L->plane;
    const RatesC<float> r = L->r;
    for (int k = 0; k < u.w; ++k) row4<S, StridedPlanes<S>, NC>(pa, g, r, u.z + 4 * lane, u.y + k, lane);
}

// One member's descriptor in the per-step launch's parameter.
struct GridLat {
    Geom g;
    const void *pop0;
    const void *pop1;
    long long plane;
    int flip;
    int xblocks;  // blocks per row: ceil(pitch / 512)
    RatesC<float> r;
};

struct GroupParams {
    int nlats;
    int xblocks;                // the members' largest blocks per row (grid x)
    int row0[kGroupLats + 1];   // first row of each member in the concatenation; row0[nlats] = rows
    GridLat lat[kGroupLats];
};

// One step of every member of a group. The members' rows are concatenated;
// block (xb, b) takes concatenated rows b, b + gridDim.y, ...; row r belongs to
// the member l with row0[l] <= r < row0[l + 1], and the block covers cells
// 512 xb .. 512 xb + 511 of that row, like block (xb, y) of the single-lattice
// VEC4 kernel (whose row loop this mirrors). Blocks past a member's row width
// skip its rows.
template <typename S, int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB)
    k_batch_grid(const __grid_constant__ GroupParams P, int parity) {
    const int lane = threadIdx.x & 31;
    const int x0 = ((int)blockIdx.x * kBatchThreads + (int)threadIdx.x) * 4;
    for (int row = blockIdx.y; row < P.row0[P.nlats]; row += gridDim.y) {
        int lo = 0, hi = P.nlats - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.row0[mid] <= row) lo = mid;
            else hi = mid - 1;
        }
        const GridLat &L = P.lat[lo];
        if ((int)blockIdx.x >= L.xblocks) continue;
        const int sel = (parity + L.flip) & 1;
        StridedPlanes<S> pa;
        pa.src = static_cast<const S *>(sel ? L.pop1 : L.pop0);
        pa.dst = static_cast<S *>(const_cast<void *>(sel ? L.pop0 : L.pop1));
        pa.plane = L.plane;
        const RatesC<float> r = L.r;  // into registers once per row rather than indexed loads at every use
        const Geom g = L.g;
        row4<S, StridedPlanes<S>, true>(pa, g, r, x0, row - P.row0[lo], lane);
    }
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

// nsteps steps of every member in one cooperative launch; the loads use the
// L2-coherent path because step s + 1 reads what step s wrote.
template <typename S, int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB)
    k_batch_persistent(const BatchLat *lats, const int4 *units, int nunits, int parity0, int nsteps, unsigned expected,
                       unsigned *bar,
                       int *status) {
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * kBatchWarps;
    for (int s = 0; s < nsteps; ++s) {
        for (int w = blockIdx.x * kBatchWarps + (threadIdx.x >> 5); w < nunits; w += stride)
            batch_unit<S, false>(lats, units[w], parity0 + s, lane);
        if (s + 1 < nsteps && !grid_barrier(bar, status, expected)) return;
    }
}

template <typename S, int MINB>
cudaError_t launch_grid_shape(const GroupParams &G, int parity, cudaStream_t st) {
    const int rows = G.row0[G.nlats];
    if (rows == 0 || G.xblocks == 0) return cudaSuccess;
    const dim3 grid(G.xblocks, rows < 65535 ? rows : 65535);
    k_batch_grid<S, MINB><<<grid, kBatchThreads, 0, st>>>(G, parity);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_batch_grid(int config, const GroupParams &G, int parity, cudaStream_t st) {
    switch (config) {
        case 1: return launch_grid_shape<S, 5>(G, parity, st);
        case 2: return launch_grid_shape<S, 6>(G, parity, st);
        case 3: return launch_grid_shape<S, 7>(G, parity, st);
        case 4: return launch_grid_shape<S, 8>(G, parity, st);
        default: return launch_grid_shape<S, 4>(G, parity, st);
    }
}

template <typename S, int MINB>
cudaError_t launch_persistent_shape(const BatchLat *lats, const int4 *units, int nunits, int parity, int nsteps,
                                    int barrier_extra, unsigned *bar, int *status, cudaStream_t st) {
    auto kern = k_batch_persistent<S, MINB>;
    int blocks = 0;
    cudaError_t e = resident_grid<GridTag<S, MINB, true>>(kern, &blocks);
    if (e != cudaSuccess) return e;
    const int need = (nunits + kBatchWarps - 1) / kBatchWarps;
    if (blocks > need) blocks = std::max(1, need);
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
    return cudaLaunchKernelEx(&cfg, kern, lats, units, nunits, parity, nsteps, expected, bar, status);
}

template <typename S>
cudaError_t launch_batch_persistent(int config, const BatchLat *lats, const int4 *units, int nunits, int parity,
                                    int nsteps, int barrier_extra, unsigned *bar, int *status, cudaStream_t st) {
    if (nunits == 0) return cudaSuccess;
    switch (config) {
        case 1: return launch_persistent_shape<S, 5>(lats, units, nunits, parity, nsteps, barrier_extra, bar, status, st);
        case 2: return launch_persistent_shape<S, 6>(lats, units, nunits, parity, nsteps, barrier_extra, bar, status, st);
        case 3: return launch_persistent_shape<S, 7>(lats, units, nunits, parity, nsteps, barrier_extra, bar, status, st);
        case 4: return launch_persistent_shape<S, 8>(lats, units, nunits, parity, nsteps, barrier_extra, bar, status, st);
        default: return launch_persistent_shape<S, 4>(lats, units, nunits, parity, nsteps, barrier_extra, bar, status, st);
    }
}

}  // namespace nomrt

using nomrt::BatchLat;

struct lbm_batch {
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only for graph capture
    int storage = -1;
    std::vector<lbm_lattice *> members;
    std::vector<int> flip;
    int64_t s = 0;  // batch steps taken
    // device buffers (allocated by the batch)
    BatchLat *d_lats = nullptr;
    int4 *d_units = nullptr;
    unsigned *d_bar = nullptr;
    int *d_status = nullptr;
    size_t cap_lats = 0, cap_units = 0;
    int nunits = 0;
    std::vector<nomrt::GroupParams> groups;  // per-step launch parameters, kGroupLats members each
    int64_t cells = 0;
    bool dirty = true;
    int config = -1;  // -1: default per storage
    int steps_per_launch = 1;
    int graph_steps = 32;
    int rows_per_unit = 1;
    int barrier_extra = 0;  // test hook: grid-barrier arrivals that never come
    int kind = LBM_BATCH_FUSED;
    // concurrent kind: one stream per member for the fork/join of the graph
    std::vector<cudaStream_t> lstreams;
    std::vector<cudaEvent_t> levents;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::string err;

    int cfg() const { return config >= 0 ? config : (storage == LBM_F16_SHIFTED ? 3 : 1); }
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

// Rebuild the device descriptors and the work list after a membership change.
lbm_status rebuild(lbm_batch *b) {
    if (!b->dirty) return LBM_OK;
    drop_graph(b);
    std::vector<BatchLat> lats(b->members.size());
    std::vector<int4> units;
    b->cells = 0;
    b->groups.clear();
    for (size_t l = 0; l < b->members.size(); ++l) {
        lbm_lattice *h = b->members[l];
        const nomrt::KParams &kp = h->kp;
        BatchLat &d = lats[l];
        d.pop0 = kp.pop[0];
        d.pop1 = kp.pop[1];
        d.plane = (long long)kp.plane;
        d.mask = kp.mask;
        d.flags = kp.flags;
        d.walls = kp.walls;
        d.nx = kp.nx;
        d.ny = kp.ny;
        d.pitch = kp.pitch;
        d.px = kp.px;
        d.py = kp.py;
        d.flip = b->flip[l];
        d.r = nomrt::make_rates<float>(kp);
        b->cells += h->fluid;
        // the per-step launch: member l joins group l / kGroupLats with its VEC4 grid
        if (l % nomrt::kGroupLats == 0) {
            b->groups.emplace_back();
            std::memset(&b->groups.back(), 0, sizeof(nomrt::GroupParams));
        }
        nomrt::GroupParams &G = b->groups.back();
        nomrt::GridLat &gl = G.lat[G.nlats];
        gl.g = nomrt::make_geom(kp);
        gl.pop0 = kp.pop[0];
        gl.pop1 = kp.pop[1];
        gl.plane = (long long)kp.plane;
        gl.flip = b->flip[l];
        gl.xblocks = (kp.pitch / 4 + nomrt::kBatchThreads - 1) / nomrt::kBatchThreads;
        gl.r = d.r;
        G.row0[G.nlats + 1] = G.row0[G.nlats] + kp.ny;
        G.xblocks = std::max(G.xblocks, gl.xblocks);
        G.nlats += 1;
        // units: runs of up to rows_per_unit consecutive rows of a 128-cell segment,
        // skipping rows of the segment that hold no fluid cell
        const int R = b->rows_per_unit;
        for (int y0 = 0; y0 < kp.ny; y0 += R)
            for (int xs = 0; xs < kp.pitch; xs += 128) {
                int first = -1, last = -1;
                for (int y = y0; y < std::min(y0 + R, kp.ny); ++y) {
                    bool any = false;
                    for (int x = xs; x < std::min(xs + 128, kp.nx) && !any; ++x)
                        any = h->flags[(size_t)y * kp.nx + x] == 0;
                    if (any) {
                        if (first < 0) first = y;
                        last = y;
                    }
                }
                if (first >= 0) units.push_back(make_int4((int)l, first, xs, last - first + 1));
            }
    }
    auto grow = [&](void **p, size_t *capacity, size_t need, size_t elem) -> cudaError_t {
        if (need <= *capacity) return cudaSuccess;
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return e;
        if (*p) cudaFree(*p);
        *p = nullptr;
        *capacity = 0;
        const size_t n = std::max(need, (size_t)64) * 3 / 2;
        e = cudaMalloc(p, n * elem);
        if (e != cudaSuccess) return e;
        *capacity = n;
        return cudaSuccess;
    };
    cudaError_t e = grow(reinterpret_cast<void **>(&b->d_lats), &b->cap_lats, lats.size(), sizeof(BatchLat));
    if (e != cudaSuccess) return bcuda(b, e, "batch descriptor allocation");
    e = grow(reinterpret_cast<void **>(&b->d_units), &b->cap_units, units.size(), sizeof(int4));
    if (e != cudaSuccess) return bcuda(b, e, "batch work list allocation");
    if (!lats.empty()) {
        e = cudaMemcpyAsync(b->d_lats, lats.data(), lats.size() * sizeof(BatchLat), cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "upload descriptors");
    }
    if (!units.empty()) {
        e = cudaMemcpyAsync(b->d_units, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "upload work list");
    }
    // the host vectors are about to go away: wait for the copies
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "upload sync");
    b->nunits = (int)units.size();
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
// `st`, so the members' kernels can run concurrently. src_fixed >= 0 re-runs
// the current step n times without advancing (tuning).
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
        for (int k = 0; k < n; ++k) {
            e = h->L->step(h->kp, cur, ls);
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

// The persistent kernel keeps its per-lattice descriptors in registers; four
// resident blocks per SM is its only shape that does not spill.
constexpr int kPersistentConfig = 0;

cudaError_t launch_steps(lbm_batch *b, int parity, int n, cudaStream_t st) {
    if (b->kind == LBM_BATCH_CONCURRENT) return launch_concurrent(b, n, st, true);
    const bool nee = any_nee(b);
    // n steps starting at parity: one launch per step, or persistent launches of steps_per_launch
    // (members with NEE walls need a pass between steps, so they force one launch per step)
    while (n > 0) {
        cudaError_t e;
        if (b->steps_per_launch > 1 && !nee) {
            const int k = std::min(n, b->steps_per_launch);
            e = b->storage == LBM_F16_SHIFTED
                    ? nomrt::launch_batch_persistent<__half>(kPersistentConfig, b->d_lats, b->d_units, b->nunits, parity, k,
                                                             b->barrier_extra, b->d_bar, b->d_status, st)
                    : nomrt::launch_batch_persistent<float>(kPersistentConfig, b->d_lats, b->d_units, b->nunits, parity, k,
                                                            b->barrier_extra, b->d_bar, b->d_status, st);
            parity = (parity + k) & 1;
            n -= k;
        } else {
            e = launch_grid_step(b, b->cfg(), parity, st);
            if (e == cudaSuccess && nee) e = launch_nee_passes(b, parity, st);
            parity ^= 1;
            n -= 1;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

lbm_status ensure_graph(lbm_batch *b) {
    if (b->graph || b->graph_steps <= 0) return LBM_OK;
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
    if (e == cudaSuccess) e = cudaMalloc(&b->d_bar, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_bar, 0, 2 * sizeof(unsigned));
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
    if (kind != LBM_BATCH_FUSED && kind != LBM_BATCH_CONCURRENT) return bfail(b, LBM_EINVAL, "unknown batch kind");
    b->kind = kind;
    drop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_set_config(lbm_batch *b, int32_t config, int32_t rows_per_unit) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (config < -1 || config >= nomrt::kBatchConfigs) return bfail(b, LBM_EINVAL, "config out of range");
    if (rows_per_unit < 1 || rows_per_unit > 1024) return bfail(b, LBM_EINVAL, "rows_per_unit must be 1..1024");
    b->config = config;
    if (rows_per_unit != b->rows_per_unit) {
        b->rows_per_unit = rows_per_unit;
        b->dirty = true;
    }
    drop_graph(b);
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
        cudaMemset(b->d_bar, 0, 2 * sizeof(unsigned));
        return bfail(b, LBM_ETIMEOUT, "the persistent batch kernel gave up a grid barrier");
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

lbm_status lbm_batch_tune(lbm_batch *b, int32_t trial_launches, int32_t *best_config, int32_t *best_rows,
                          float *ms_per_launch) {
    if (!b) return bfail(nullptr, LBM_EINVAL, "batch is NULL");
    if (trial_launches < 1) return bfail(b, LBM_EINVAL, "trial_launches must be >= 1");
    if (b->members.empty()) return bfail(b, LBM_EINVAL, "batch is empty");
    // Each trial re-runs the current step with the same source parity: it
    // rewrites the destination buffers with the same values and leaves the
    // state the next real step reads untouched.
    const int parity = (int)(b->s & 1);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, LBM_ECUDA, "event create");
    int best = 0;
    float best_ms = 1e30f;
    lbm_status out = rebuild(b);
    for (int c = 0; c < nomrt::kBatchConfigs && out == LBM_OK; ++c) {
        auto run = [&](int n) -> cudaError_t {
            for (int k = 0; k < n; ++k) {
                cudaError_t e = launch_grid_step(b, c, parity, b->stream);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        };
        cudaError_t e = run(1);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = run(trial_launches);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            out = bcuda(b, e, "tuning launch");
            break;
        }
        ms /= (float)trial_launches;
        if (ms_per_launch) ms_per_launch[c] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    // the concurrent kind: every member's own kernel, members in parallel
    float conc_ms = 1e30f;
    if (out == LBM_OK) {
        cudaError_t e = launch_concurrent(b, 1, b->stream, false);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = launch_concurrent(b, trial_launches, b->stream, false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&conc_ms, e0, e1);
        if (e != cudaSuccess) out = bcuda(b, e, "tuning launch (concurrent)");
        conc_ms /= (float)trial_launches;
        if (ms_per_launch) ms_per_launch[nomrt::kBatchConfigs] = conc_ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (out != LBM_OK) return out;
    b->kind = conc_ms < best_ms ? LBM_BATCH_CONCURRENT : LBM_BATCH_FUSED;
    b->config = best;
    drop_graph(b);
    if (best_config) *best_config = b->kind == LBM_BATCH_CONCURRENT ? -2 : best;
    if (best_rows) *best_rows = b->rows_per_unit;
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
    if (config) *config = b->kind == LBM_BATCH_CONCURRENT ? -2 : b->cfg();
    if (rows_per_unit) *rows_per_unit = b->rows_per_unit;
    if (steps_done) *steps_done = b->s;
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
    if (b->d_lats) cudaFree(b->d_lats);
    if (b->d_units) cudaFree(b->d_units);
    if (b->d_bar) cudaFree(b->d_bar);
    if (b->d_status) cudaFree(b->d_status);
    delete b;
}

}  // extern "C"
