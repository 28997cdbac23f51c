// Host side of the C ABI declared in include/nomrt_lbm.h: parameter
// validation, device-memory layout, uploads, the step loop and the
// synchronising read-outs. The arithmetic of the method runs in the kernels
// of nomrt_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "lattice_impl.h"
#include "nomrt_internal.h"
#include "nomrt_lbm.h"

using nomrt::KParams;
using nomrt::Layout;
using nomrt::kSolid;
using nomrt::WallDev;

namespace {

thread_local std::string g_create_error;

constexpr double kCs2 = 1.0 / 3.0;  // D2Q9 c_s^2 (Sec. 2.1)
constexpr size_t kAlign = 256;
constexpr size_t kStageBytes = 16u << 20;  // row-chunked host transfers

const int kEx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};  // Eq. 5
const int kEy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__constant__ int kExD[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kEyD[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
const double kW[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t elem_bytes(int storage) { return storage == LBM_F64 ? 8 : storage == LBM_F32_SHIFTED ? 4 : 2; }

int thermal_q(const lbm_params *p) { return p->thermal_q == 9 ? 9 : 5; }

Layout make_layout(int nx, int ny, int storage, int n_walls, int n_nee, int tq) {
    Layout L;
    const size_t eb = elem_bytes(storage);
    L.nq = 9 + tq;
    L.pitch = (int)align_up((size_t)nx, 128 / eb);
    L.plane = (size_t)ny * L.pitch;
    L.pop_bytes = align_up(L.plane * eb * L.nq, kAlign);
    size_t o = 0;
    L.off_pop[0] = o; o += L.pop_bytes;
    L.off_pop[1] = o; o += L.pop_bytes;
    L.off_mask = o; o += align_up(L.plane, kAlign);
    L.off_flags = o; o += align_up(L.plane, kAlign);
    L.off_walls = o; o += align_up(sizeof(WallDev) * (size_t)(n_walls + 1), kAlign);
    L.off_snap = o; o += align_up(3 * L.plane * sizeof(double), kAlign);
    const size_t row_bytes = (size_t)L.nq * nx * sizeof(double);
    // at most 8192 rows per chunk keeps every chunked launch under the 65535 grid-y limit
    L.stage_rows = (int)std::max<size_t>(1, std::min<size_t>({(size_t)ny, kStageBytes / row_bytes, (size_t)8192}));
    L.off_stage = o; o += align_up(row_bytes * L.stage_rows, kAlign);
    L.off_part = o; o += align_up(sizeof(double) * nomrt::kRedBlocks * 8, kAlign);
    L.off_res = o; o += align_up(sizeof(double) * 8, kAlign);
    L.off_status = o; o += kAlign;
    L.off_nee_dir = o; o += align_up(L.plane, kAlign);
    L.off_nee = o; o += align_up(sizeof(int2) * (size_t)std::max(1, n_nee), kAlign);
    L.total = o;
    return L;
}

struct Derived {
    double s_nu, z_a;
};

// Rates from the transport coefficients: nu = c_s^2 (1/s_nu - 1/2) (Sec. 2.1),
// alpha = c_sT^2 (1/zeta_alpha - 1/2) with c_sT^2 = varpi/2 (Sec. 2.2), or
// c_sT^2 = c_s^2 for the D2Q9 temperature model (Eq. 33).
Derived derive(const lbm_params *p) {
    Derived d;
    d.s_nu = 1.0 / (0.5 + p->nu / kCs2);
    const double csT2 = thermal_q(p) == 9 ? kCs2 : 0.5 * p->varpi;
    d.z_a = 1.0 / (0.5 + p->alpha / csT2);
    return d;
}

bool in_open_02(double v) { return std::isfinite(v) && v > 0.0 && v < 2.0; }

// Direction i of a boundary node's nearest fluid node x + e_i: an axis
// neighbour if one is fluid, else a diagonal one; 0 if there is none.
int nee_direction(const lbm_params *p, int x, int y) {
    for (int i = 1; i < 9; ++i) {
        int sx = x + kEx[i], sy = y + kEy[i];
        if (p->periodic_x) sx = (sx + p->nx) % p->nx;
        if (p->periodic_y) sy = (sy + p->ny) % p->ny;
        if (sx < 0 || sx >= p->nx || sy < 0 || sy >= p->ny) continue;
        if (p->flags[(size_t)sy * p->nx + sx] == 0) return i;
    }
    return 0;
}

// One pass over the cells: validates the flag map and, if `out` is given,
// builds the device-side maps. Rows are split into bands scanned by host
// threads; results are merged in row order, so they do not depend on the
// thread count.
struct CellScan {
    int pitch = 0;
    uint8_t *mask = nullptr;   // ny * pitch link map (bit i-1: direction i pulls from a solid cell; 0xFF
                               // for solid cells and the padding columns)
    uint8_t *flags = nullptr;  // ny * pitch wall ids (0 in the padding columns)
};

struct ScanResult {
    std::string err;  // empty if valid
    int64_t fluid = 0;
    std::vector<int2> nee;  // (cell offset in the pitched layout, direction | wall id << 8)
};

// Row y, cell by cell, in row-major order: the exact reference for the fast
// path below, and the path that produces the error message of a row holding
// an invalid cell. Returns false at the row's first invalid cell.
bool scan_row_exact(const lbm_params *p, const uint8_t *halfway, int y, const CellScan *out, ScanResult &r) {
    const int nx = p->nx, ny = p->ny;
    const bool px = p->periodic_x != 0, py = p->periodic_y != 0;
    char buf[256];
    // source rows of directions with e_y = -1, 0, +1: y + 1, y, y - 1
    const int ys[3] = {py ? (y + 1) % ny : y + 1, y, py ? (y - 1 + ny) % ny : y - 1};
    const uint8_t *row = p->flags + (size_t)y * nx;
    for (int x = 0; x < nx; ++x) {
        const uint8_t k = row[x];
        if (k > p->n_walls) {
            snprintf(buf, sizeof buf, "cell (%d, %d) has wall id %d > n_walls", x, y, (int)k);
            r.err = buf;
            return false;
        }
        const size_t off = (size_t)y * (out ? out->pitch : 0) + x;
        if (out) out->flags[off] = k;
        if (k) {
            if (!halfway[k]) {  // boundary node of a node-based wall
                const int d = nee_direction(p, x, y);
                if (d == 0) {
                    snprintf(buf, sizeof buf,
                             "boundary node (%d, %d) of an extrapolated wall has no fluid neighbour", x, y);
                    r.err = buf;
                    return false;
                }
                r.nee.push_back(out ? make_int2((int)off, d | ((int)k << 8)) : make_int2(0, 0));
            }
            continue;
        }
        unsigned m = 0;
        for (int i = 1; i < 9; ++i) {
            int sx = x - kEx[i];
            if (px) sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
            const int sy = ys[kEy[i] + 1];
            if (sx < 0 || sx >= nx || sy < 0 || sy >= ny) {
                snprintf(buf, sizeof buf,
                         "fluid cell (%d, %d) touches a non-periodic edge; add a frame of solid cells", x, y);
                r.err = buf;
                return false;
            }
            if (halfway[p->flags[(size_t)sy * nx + sx]]) m |= 1u << (i - 1);
        }
        if (m == 0xFFu) {
            snprintf(buf, sizeof buf, "fluid cell (%d, %d) has no fluid neighbour", x, y);
            r.err = buf;
            return false;
        }
        ++r.fluid;
        if (out) out->mask[off] = (uint8_t)m;
    }
    return true;
}

// Cell kinds of row y, padded by one cell on each side: 1 = solid (a
// bounce-back wall), 0 = fluid or a boundary node, 2 = outside the domain
// (a non-periodic edge), 4 = a wall id above n_walls.
void kinds_row(const lbm_params *p, const uint8_t *halfway, bool all_halfway, int y, uint8_t *pad) {
    const int nx = p->nx, ny = p->ny;
    if (y < 0 || y >= ny) {
        if (!p->periodic_y) {
            std::memset(pad, 2, (size_t)nx + 2);
            return;
        }
        y = (y + ny) % ny;
    }
    const uint8_t *__restrict row = p->flags + (size_t)y * nx;
    uint8_t *__restrict out = pad + 1;
    const uint8_t nw = (uint8_t)p->n_walls;
    if (all_halfway) {  // every wall bounces back: no table lookup, so the loop vectorises
        for (int x = 0; x < nx; ++x) out[x] = row[x] > nw ? 4 : (row[x] != 0 ? 1 : 0);
    } else {
        for (int x = 0; x < nx; ++x) out[x] = row[x] > nw ? 4 : halfway[row[x]];
    }
    pad[0] = p->periodic_x ? pad[nx] : 2;
    pad[nx + 1] = p->periodic_x ? pad[1] : 2;
}

// Rows [y0, y1). Stops at the band's first invalid cell (row-major order).
// Each row is scanned from three padded rows of cell kinds in a loop without
// branches (it vectorises); a row holding an invalid cell (a bad wall id, a
// fluid cell at a non-periodic edge or without a fluid neighbour, a boundary
// node without a fluid neighbour) is rescanned by scan_row_exact, which names
// the first one.
void scan_rows(const lbm_params *p, const uint8_t *halfway, bool all_halfway, int y0, int y1, const CellScan *out,
               ScanResult &r) {
    const int nx = p->nx;
    std::vector<uint8_t> buf(4 * ((size_t)nx + 2));
    uint8_t *up = buf.data(), *mid = up + nx + 2, *dn = mid + nx + 2;  // rows y + 1, y, y - 1
    uint8_t *const mrow = dn + nx + 2;
    if (y0 < y1) {
        kinds_row(p, halfway, all_halfway, y0 - 1, dn);
        kinds_row(p, halfway, all_halfway, y0, mid);
    }
    for (int y = y0; y < y1; ++y) {
        kinds_row(p, halfway, all_halfway, y + 1, up);
        const uint8_t *__restrict row = p->flags + (size_t)y * nx;
        const uint8_t *__restrict U = up;
        const uint8_t *__restrict C = mid;
        const uint8_t *__restrict D = dn;
        uint8_t *__restrict M = mrow;
        // bit 1: a fluid cell pulls from outside; bit 2: a bad wall id; bit 3: a fluid
        // cell without a fluid neighbour; bit 4: a boundary node of a node-based wall
        uint8_t odd = 0;
        int fluid = 0;
        for (int x = 0; x < nx; ++x) {
            const uint8_t w = C[x], c = C[x + 1], e = C[x + 2];
            const uint8_t sw = D[x], s = D[x + 1], se = D[x + 2];
            const uint8_t nw = U[x], n = U[x + 1], ne = U[x + 2];
            // bit i-1: the source x - e_i of direction i is not fluid
            const uint8_t m = (uint8_t)((w ? 1 : 0) | (s ? 2 : 0) | (e ? 4 : 0) | (n ? 8 : 0) | (sw ? 16 : 0) |
                                        (se ? 32 : 0) | (ne ? 64 : 0) | (nw ? 128 : 0));
            const uint8_t fm = row[x] == 0 ? 0xFF : 0;  // all ones for a fluid cell
            const uint8_t all = (uint8_t)(w | s | e | n | sw | se | ne | nw);
            const uint8_t full = m == 0xFF ? 8 : 0;
            const uint8_t node = (row[x] != 0 && c == 0) ? 16 : 0;
            odd |= (uint8_t)((c & 4) | ((all & 2) & fm) | (full & fm) | node);
            fluid += fm & 1;
            M[x] = (uint8_t)(m | ~fm);  // kSolid for every cell that is not fluid
        }
        const bool nodes = (odd & 16) != 0;
        odd &= 15;
        const size_t base = (size_t)y * (out ? out->pitch : 0);
        if (out) {
            std::memcpy(out->flags + base, row, (size_t)nx);
            std::memcpy(out->mask + base, mrow, (size_t)nx);
            std::memset(out->flags + base + nx, 0, (size_t)(out->pitch - nx));
            std::memset(out->mask + base + nx, kSolid, (size_t)(out->pitch - nx));
        }
        const size_t nee0 = r.nee.size();
        if (nodes && !odd) {
            for (int x = 0; x < nx; ++x) {
                if (row[x] == 0 || mid[x + 1] != 0) continue;
                const int d = nee_direction(p, x, y);
                if (d == 0) {
                    odd = 8;
                    break;
                }
                r.nee.push_back(out ? make_int2((int)(base + x), d | ((int)row[x] << 8)) : make_int2(0, 0));
            }
        }
        if (odd) {
            r.nee.resize(nee0);
            if (!scan_row_exact(p, halfway, y, out, r)) return;
        } else {
            r.fluid += fluid;
        }
        uint8_t *t = dn;
        dn = mid;
        mid = up;
        up = t;
    }
}

ScanResult scan_cells(const lbm_params *p, const CellScan *out) {
    uint8_t halfway[256] = {0};  // wall id -> its cells are solid (HALFWAY)
    bool all_halfway = true;
    for (int k = 1; k <= p->n_walls; ++k) {
        halfway[k] = p->walls[k - 1].scheme == LBM_WALL_HALFWAY;
        all_halfway = all_halfway && halfway[k];
    }
    const size_t cells = (size_t)p->nx * p->ny;
    unsigned hw = std::thread::hardware_concurrency();
    int nthreads = (int)std::min<size_t>(std::max(1u, std::min(hw, 16u)), std::max<size_t>(1, cells >> 18));
    nthreads = std::min(nthreads, p->ny);
    std::vector<ScanResult> part(nthreads);
    std::vector<std::thread> pool;
    const int band = (p->ny + nthreads - 1) / nthreads;
    for (int t = 1; t < nthreads; ++t)
        pool.emplace_back(scan_rows, p, halfway, all_halfway, std::min(p->ny, t * band),
                          std::min(p->ny, (t + 1) * band), out, std::ref(part[t]));
    scan_rows(p, halfway, all_halfway, 0, std::min(p->ny, band), out, part[0]);
    for (auto &th : pool) th.join();
    ScanResult r;
    for (auto &q : part) {
        if (!q.err.empty()) {
            r.err = q.err;  // the first band with an error holds the first invalid cell
            return r;
        }
        r.fluid += q.fluid;
        r.nee.insert(r.nee.end(), q.nee.begin(), q.nee.end());
    }
    return r;
}

// Returns an empty string if p's scalar fields are valid, else the reason
// (the flag map is checked by scan_cells).
std::string validate(const lbm_params *p) {
    char buf[256];
    if (!p) return "params is NULL";
    if (p->nx < 1 || p->ny < 1) return "nx and ny must be >= 1";
    if (!p->flags) return "flags is NULL";
    if (p->n_walls < 0 || p->n_walls > 254) return "n_walls must be in 0..254";
    if (p->n_walls > 0 && !p->walls) return "walls is NULL";
    if (p->storage < LBM_F64 || p->storage > LBM_F16_SHIFTED) return "unknown storage";
    if (!(std::isfinite(p->varpi) && p->varpi > 0.0 && p->varpi < 1.0)) return "varpi must be in (0, 1)";
    if (!(std::isfinite(p->nu) && p->nu > 0.0)) return "nu must be > 0";
    if (!(std::isfinite(p->alpha) && p->alpha > 0.0)) return "alpha must be > 0";
    if (p->thermal_q != 0 && p->thermal_q != 5 && p->thermal_q != 9) return "thermal_q must be 0, 5 or 9";
    if (p->collision != LBM_COLLISION_MRT && p->collision != LBM_COLLISION_BGK) return "unknown collision operator";
    if (thermal_q(p) == 9) {
        if (!in_open_02(p->zeta_q) || !in_open_02(p->zeta_eps)) return "zeta_q and zeta_eps must be in (0, 2)";
        if (!std::isfinite(p->theta)) return "theta must be finite";
    }
    Derived d = derive(p);
    const double rates[7] = {d.s_nu, p->s_e, p->s_q, p->s_eps, d.z_a, p->zeta_e, p->zeta_nu};
    const char *names[7] = {"s_nu", "s_e", "s_q", "s_eps", "zeta_alpha", "zeta_e", "zeta_nu"};
    for (int k = 0; k < 7; ++k)
        if (!in_open_02(rates[k])) {
            snprintf(buf, sizeof buf, "rate %s = %g is outside (0, 2)", names[k], rates[k]);
            return buf;
        }
    const double finite[6] = {p->g_beta, p->T0, p->ax, p->ay, 0, 0};
    for (double v : finite)
        if (!std::isfinite(v)) return "g_beta, T0, ax, ay must be finite";
    for (int k = 0; k < p->n_walls; ++k) {
        const lbm_wall &w = p->walls[k];
        if (!std::isfinite(w.ux) || !std::isfinite(w.uy) || !std::isfinite(w.T)) return "wall values must be finite";
        if (w.kind != LBM_T_DIRICHLET && w.kind != LBM_T_ADIABATIC) return "unknown wall thermal kind";
        if (w.scheme != LBM_WALL_HALFWAY && w.scheme != LBM_WALL_NEE) return "unknown wall scheme";
    }
    const size_t eb = elem_bytes(p->storage);
    const size_t pitch = align_up((size_t)p->nx, 128 / eb);
    if ((size_t)p->ny * pitch >= (size_t)INT32_MAX) return "lattice too large (ny * pitch must be < 2^31)";
    return std::string();
}

const nomrt::Launchers &launchers_for(int storage) {
    return storage == LBM_F64 ? nomrt::launchers_f64()
           : storage == LBM_F32_SHIFTED ? nomrt::launchers_f32()
                                        : nomrt::launchers_f16();
}

}  // namespace

void nomrt::set_thread_error(const char *msg) { g_create_error = msg; }



namespace {

lbm_status fail(lbm_lattice *h, lbm_status st, const std::string &msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return st;
}

lbm_status cuda_fail(lbm_lattice *h, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, LBM_ECUDA, m);
}

#define LBM_CUDA(h, call, what)                      \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

// After a stream synchronisation: a kernel that gave up a bounded wait left a
// non-zero status word, or (bounds-checking build) a refused access left a
// non-zero bounds word; report it once and clear both.
lbm_status check_status(lbm_lattice *h) {
    int st[2] = {0, 0};
    cudaError_t e = cudaMemcpy(st, h->kp.status, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "read status");
    if (st[0] == nomrt::kStatusOk && st[1] == 0) return LBM_OK;
    const int zero[2] = {0, 0};
    e = cudaMemcpy(h->kp.status, zero, sizeof zero, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "clear status");
    if (st[1] != 0) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "bounds-checking build: an index check failed at site %d (the access was skipped; the state is "
                 "invalid)", st[1]);
        return fail(h, LBM_ECUDA, buf);
    }
    return fail(h, LBM_ETIMEOUT, "a kernel gave up a bounded wait (device status word set)");
}

#define LBM_STATUS(h)                      \
    do {                                   \
        lbm_status s_ = check_status(h);   \
        if (s_ != LBM_OK) return s_;       \
    } while (0)

// Steps per replayed graph: a long one and a short one (both even: a graph starts and ends on
// buffer 0), so that runs from kGraphShort steps up replay graphs.
constexpr int kGraphSteps = 32;
constexpr int kGraphShort = 4;

void drop_graph(lbm_lattice *h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->graph_short) cudaGraphExecDestroy(h->graph_short);
    h->graph = nullptr;
    h->graph_short = nullptr;
}

// Captures `steps` steps starting from buffer 0 on a private stream (the lattice's own stream
// may be the legacy default stream, which cannot be captured; the graph launches on any
// stream). nullptr on failure (the error is cleared).
cudaGraphExec_t capture_steps(lbm_lattice *h, int steps) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    bool ok = h->cap_stream || cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) ok = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        for (int s = 0; s < steps && ok; ++s) ok = h->L->step(h->kp, s & 1, h->cap_stream) == cudaSuccess;
        ok = (cudaStreamEndCapture(h->cap_stream, &g) == cudaSuccess) && ok && g;
    }
    if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        if (ge) cudaGraphExecDestroy(ge);
        cudaGetLastError();
        return nullptr;
    }
    return ge;
}

// Both graphs for the current kernel choice; on any failure the lattice falls back to
// direct launches for good.
void capture_graph(lbm_lattice *h) {
    h->graph = capture_steps(h, kGraphSteps);
    h->graph_short = h->graph ? capture_steps(h, kGraphShort) : nullptr;
    if (!h->graph || !h->graph_short) {
        drop_graph(h);
        h->graph_off = true;
        return;
    }
    h->graph_variant = h->kp.variant;
    h->graph_config = h->kp.config;
}

lbm_status step_direct(lbm_lattice *h, int64_t n) {
    for (int64_t s = 0; s < n; ++s) {
        cudaError_t e = h->L->step(h->kp, h->cur, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
        h->cur ^= 1;
        ++h->steps;
    }
    if (n > 0) h->direct_done = true;
    return LBM_OK;
}

// The device-side maps of a lattice whose walls are all halfway (no node-based
// wall, so the layout does not depend on the flag map): one thread per cell of
// the pitched layout reads the wall ids of the cell and of its eight pull
// sources from `src` (row stride src_stride; the pitched flag plane itself,
// or the caller's raw map read in place), and writes the pitched flag plane
// (copy = 1), the link map (bit i-1: direction i pulls from a solid cell;
// 0xFF for solid cells and the padding columns) and a zero boundary-node
// direction. Validation as the host scan: a wall id above n_walls, a fluid
// cell pulling from beyond a non-periodic edge, a fluid cell with no fluid
// neighbour; the lowest such cell index (row-major) goes to *first_bad, and the
// fluid cells are counted into *fluid.
__global__ void __launch_bounds__(256) k_build_maps(const uint8_t *src, long long src_stride, int copy, int nx, int ny,
                                                    int y0, int pitch, int px, int py, int n_walls, uint8_t *flags,
                                                    uint8_t *mask, uint8_t *nee_dir,
                                                    unsigned long long *first_bad, unsigned long long *fluid) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = y0 + (int)blockIdx.y;  // rows y0 .. y0 + gridDim.y - 1 of the whole lattice
    __shared__ unsigned count;
    if (threadIdx.x == 0) count = 0;
    __syncthreads();
    if (x < pitch && y < ny) {
        const size_t off = (size_t)y * pitch + x;
        uint8_t m = nomrt::kSolid;
        uint8_t k = 0;
        if (x < nx) {
            k = src[(long long)y * src_stride + x];
            bool bad = k > n_walls;
            if (k == 0) {
                unsigned bits = 0;
                for (int i = 1; i < 9; ++i) {
                    int sx = x - kExD[i], sy = y - kEyD[i];
                    if (px) sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
                    if (py) sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                    if (sx < 0 || sx >= nx || sy < 0 || sy >= ny) {
                        bad = true;
                        break;
                    }
                    if (src[(long long)sy * src_stride + sx] != 0) bits |= 1u << (i - 1);
                }
                bad = bad || bits == 0xFFu;
                m = (uint8_t)bits;
                if (!bad) atomicAdd(&count, 1u);
            }
            if (bad) atomicMin(first_bad, (unsigned long long)y * (unsigned long long)nx + (unsigned long long)x);
        }
        if (copy) flags[off] = k;
        else if (x >= nx) flags[off] = 0;
        mask[off] = m;
        nee_dir[off] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0 && count) atomicAdd(fluid, (unsigned long long)count);
}

// A device address through which the GPU reads `p` in place (page-locked or
// registered host memory, managed or device memory), or nullptr for ordinary
// pageable host memory.
const void *device_view(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged || a.type == cudaMemoryTypeDevice)
        return a.devicePointer;
    return nullptr;
}

bool all_walls_halfway(const lbm_params *p) {
    for (int k = 0; k < p->n_walls; ++k)
        if (p->walls[k].scheme != LBM_WALL_HALFWAY) return false;
    return true;
}

// Fluid cells of the middle line across the lattice along the normal of `side`
// (the default length of lbm_nusselt).
void middle_lines(const lbm_params *p, int *across_x, int *across_y) {
    int cx = 0, cy = 0;
    const int y = p->ny / 2, x = p->nx / 2;
    for (int i = 0; i < p->nx; ++i) cx += p->flags[(size_t)y * p->nx + i] == 0;
    for (int j = 0; j < p->ny; ++j) cy += p->flags[(size_t)j * p->nx + x] == 0;
    *across_x = cx;
    *across_y = cy;
}

}  // namespace

extern "C" {

lbm_status lbm_validate(const lbm_params *p) {
    std::string why = validate(p);
    if (!why.empty()) return fail(nullptr, LBM_EINVAL, why);
    ScanResult sr = scan_cells(p, nullptr);
    if (!sr.err.empty()) return fail(nullptr, LBM_EINVAL, sr.err);
    return LBM_OK;
}

size_t lbm_footprint_bytes(const lbm_params *p) {
    std::string why = validate(p);
    if (!why.empty()) {
        g_create_error = why;
        return 0;
    }
    int n_nee = 0;
    if (!all_walls_halfway(p)) {  // the boundary nodes of node-based walls take space: count them
        ScanResult sr = scan_cells(p, nullptr);
        if (!sr.err.empty()) {
            g_create_error = sr.err;
            return 0;
        }
        n_nee = (int)sr.nee.size();
    }
    return make_layout(p->nx, p->ny, p->storage, p->n_walls, n_nee, thermal_q(p)).total;
}

lbm_status lbm_create(const lbm_params *p, void *cuda_stream, void *device_mem, size_t device_bytes,
                      lbm_lattice **out) {
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why = validate(p);
    if (!why.empty()) return fail(nullptr, LBM_EINVAL, why);
    lbm_lattice *h = new (std::nothrow) lbm_lattice();
    if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    h->nx = p->nx;
    h->ny = p->ny;
    h->px = p->periodic_x != 0;
    h->py = p->periodic_y != 0;
    h->storage = p->storage;
    h->n_walls = p->n_walls;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    const int pitch0 = (int)align_up((size_t)p->nx, 128 / elem_bytes(p->storage));
    const size_t map_bytes = (size_t)p->ny * pitch0;
    // Lattices with node-based walls: host-side maps in one pass over the cells (which also
    // validates them): wall ids, the link map (bit i-1: direction i pulls from a solid cell;
    // padding and solid cells 0xFF) and the boundary nodes. Every other lattice builds its
    // maps on the GPU (k_build_maps), from the flag map read in place when the GPU can.
    const bool gpu_maps = all_walls_halfway(p);
    std::unique_ptr<uint8_t[]> hmask, hflags;
    std::vector<int2> hnee;
    if (!gpu_maps) {
        // written in full by the scan (padding columns included), so left uninitialised here
        hmask.reset(new (std::nothrow) uint8_t[map_bytes]);
        hflags.reset(new (std::nothrow) uint8_t[map_bytes]);
        if (!hmask || !hflags) {
            lbm_destroy(h);
            return fail(nullptr, LBM_ENOMEM, "host allocation failed");
        }
        CellScan cs;
        cs.pitch = pitch0;
        cs.mask = hmask.get();
        cs.flags = hflags.get();
        ScanResult sr = scan_cells(p, &cs);
        if (!sr.err.empty()) {
            lbm_destroy(h);
            return fail(nullptr, LBM_EINVAL, sr.err);
        }
        hnee.swap(sr.nee);
        h->fluid = sr.fluid;
    }
    middle_lines(p, &h->across_x, &h->across_y);
    const int n_nee = (int)hnee.size();
    h->lay = make_layout(p->nx, p->ny, p->storage, p->n_walls, n_nee, thermal_q(p));
    h->L = &launchers_for(p->storage);
    const size_t need = h->lay.total;
    auto bail = [&](lbm_status st, const std::string &m) {
        g_create_error = m;
        lbm_destroy(h);
        return st;
    };
    if (device_mem) {
        uintptr_t a = reinterpret_cast<uintptr_t>(device_mem);
        if (a % kAlign) return bail(LBM_EINVAL, "device_mem must be 256-byte aligned");
        if (device_bytes < need) return bail(LBM_ENOMEM, "device_mem smaller than lbm_footprint_bytes");
        h->mem = static_cast<char *>(device_mem);
    } else {
        void *m = nullptr;
        cudaError_t e = cudaMalloc(&m, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bail(LBM_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
        }
        h->mem = static_cast<char *>(m);
        h->owns_mem = true;
    }

    const int nx = p->nx, ny = p->ny, pitch = h->lay.pitch;
    std::vector<WallDev> hw((size_t)p->n_walls + 1);
    std::memset(hw.data(), 0, sizeof(WallDev) * hw.size());
    const double T_ref = p->storage == LBM_F64 ? 0.0 : p->T0;
    const int tq = thermal_q(p);
    for (int k = 1; k <= p->n_walls; ++k) {
        const lbm_wall &w = p->walls[k - 1];
        for (int i = 0; i < 9; ++i) hw[k].cf[i] = 2.0 * kW[i] * 1.0 * (kEx[i] * w.ux + kEy[i] * w.uy) / kCs2;
        if (w.kind == LBM_T_DIRICHLET) {
            hw[k].tsgn = -1.0;
            hw[k].tb = 0.5 * p->varpi * (w.T - T_ref);
            // D2Q9 model: twice the even part of Eq. 31 at the wall, less the storage shift
            const double uw2 = w.ux * w.ux + w.uy * w.uy;
            for (int i = 0; i < 9; ++i) {
                const double eu = kEx[i] * w.ux + kEy[i] * w.uy;
                const double even = kW[i] * w.T * (1.0 + p->theta * (eu * eu / (2.0 * kCs2 * kCs2) - uw2 / (2.0 * kCs2)));
                hw[k].tb9[i] = 2.0 * (even - kW[i] * T_ref);
            }
        } else {
            hw[k].tsgn = 1.0;
            hw[k].tb = 0.0;
        }
        hw[k].Tw = w.T;
        hw[k].uwx = w.ux;
        hw[k].uwy = w.uy;
        hw[k].nee = w.scheme == LBM_WALL_NEE ? 1.0 : 0.0;
        hw[k].adiabatic = w.kind == LBM_T_ADIABATIC ? 1.0 : 0.0;
    }

    KParams &kp = h->kp;
    kp.nx = nx;
    kp.ny = ny;
    kp.pitch = pitch;
    kp.px = h->px;
    kp.py = h->py;
    kp.plane = h->lay.plane;
    kp.pop[0] = h->mem + h->lay.off_pop[0];
    kp.pop[1] = h->mem + h->lay.off_pop[1];
    kp.mask = reinterpret_cast<const uint8_t *>(h->mem + h->lay.off_mask);
    kp.flags = reinterpret_cast<const uint8_t *>(h->mem + h->lay.off_flags);
    kp.walls = reinterpret_cast<const WallDev *>(h->mem + h->lay.off_walls);
    Derived d = derive(p);
    kp.s_e = p->s_e;
    kp.s_nu = d.s_nu;
    kp.s_q = p->s_q;
    kp.s_eps = p->s_eps;
    kp.z_a = d.z_a;
    kp.z_e = p->zeta_e;
    kp.z_nu = p->zeta_nu;
    kp.g_beta = p->g_beta;
    kp.T0 = p->T0;
    kp.ax = p->ax;
    kp.ay = p->ay;
    kp.varpi = p->varpi;
    kp.rho_ref = p->storage == LBM_F64 ? 0.0 : 1.0;
    kp.T_ref = T_ref;
    kp.tq = tq;
    kp.theta = tq == 9 ? p->theta : 0.0;
    kp.z_q = tq == 9 ? p->zeta_q : 0.0;
    kp.z_eps = tq == 9 ? p->zeta_eps : 0.0;
    kp.bgk = p->collision == LBM_COLLISION_BGK ? 1 : 0;
    kp.nee = reinterpret_cast<const int2 *>(h->mem + h->lay.off_nee);
    kp.n_nee = (int)hnee.size();
    kp.nee_dir = reinterpret_cast<const uint8_t *>(h->mem + h->lay.off_nee_dir);
    kp.variant = nomrt::kStepAuto;
    kp.config = 0;
    kp.status = reinterpret_cast<int *>(h->mem + h->lay.off_status);
    kp.oob = kp.status + 1;  // the status slot holds 256 bytes
    kp.blk_lo = h->mem;
    kp.blk_hi = h->mem + need;

    cudaStream_t st = h->stream;
    auto cuda_bail = [&](cudaError_t e, const char *what) {
        return bail(LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
    // zeros where they must start: the status words
    if ((e = cudaMemsetAsync(h->mem + h->lay.off_status, 0, kAlign, st)) != cudaSuccess)
        return cuda_bail(e, "clear status");
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(h->result());  // first bad cell, fluid
    if (gpu_maps) {
        if ((e = cudaMemsetAsync(counters, 0xFF, sizeof(unsigned long long), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(counters + 1, 0, sizeof(unsigned long long), st)) != cudaSuccess)
            return cuda_bail(e, "clear counters");
        uint8_t *dflags = reinterpret_cast<uint8_t *>(h->mem + h->lay.off_flags);
        const uint8_t *src = static_cast<const uint8_t *>(device_view(p->flags));
        long long stride = nx;
        int copy = 1;
        if (!src) {  // pageable: copy the map into the pitched flag plane, then build in place
            if ((e = cudaMemcpy2DAsync(dflags, (size_t)pitch, p->flags, (size_t)nx, (size_t)nx, (size_t)ny,
                                       cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_bail(e, "upload flags");
            src = dflags;
            stride = pitch;
            copy = 0;
        }
        for (int y0 = 0; y0 < ny; y0 += 65535) {  // the grid's y extent is at most 65535 rows per launch
            const int rows = std::min(65535, ny - y0);
            const dim3 grid((unsigned)((pitch + 255) / 256), (unsigned)rows);
            k_build_maps<<<grid, 256, 0, st>>>(src, stride, copy, nx, ny, y0, pitch, h->px, h->py, p->n_walls, dflags,
                                              const_cast<uint8_t *>(kp.mask), const_cast<uint8_t *>(kp.nee_dir),
                                              counters, counters + 1);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_bail(e, "map kernel");
        }
    } else {
        if ((e = cudaMemsetAsync(h->mem + h->lay.off_nee_dir, 0, map_bytes, st)) != cudaSuccess)
            return cuda_bail(e, "clear boundary-node directions");
        if ((e = cudaMemcpyAsync(h->mem + h->lay.off_mask, hmask.get(), map_bytes, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return cuda_bail(e, "upload link map");
        if ((e = cudaMemcpyAsync(h->mem + h->lay.off_flags, hflags.get(), map_bytes, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return cuda_bail(e, "upload flags");
    }
    if ((e = cudaMemcpyAsync(h->mem + h->lay.off_walls, hw.data(), sizeof(WallDev) * hw.size(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_bail(e, "upload walls");
    std::vector<uint8_t> hdir;  // nearest-fluid directions of boundary nodes (the device plane is zeroed)
    if (!hnee.empty()) {
        hdir.assign(map_bytes, 0);
        for (const int2 &b : hnee) hdir[(size_t)b.x] = (uint8_t)(b.y & 0xFF);
        if ((e = cudaMemcpyAsync(h->mem + h->lay.off_nee_dir, hdir.data(), map_bytes, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return cuda_bail(e, "upload boundary-node directions");
        if ((e = cudaMemcpyAsync(h->mem + h->lay.off_nee, hnee.data(), hnee.size() * sizeof(int2),
                                 cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_bail(e, "upload boundary nodes");
    }
    // initial state (and zeros in the other buffer): T read in place when the GPU can reach it
    // (or T0 everywhere), else in row chunks through the staging area, which holds nq rows of
    // populations and so stage_rows * nq rows of T. Stream order keeps a chunk's upload behind
    // the previous chunk's init kernel; one wait at the end covers the host buffers.
    const double *Tv = p->T_init ? static_cast<const double *>(device_view(p->T_init)) : nullptr;
    if (!p->T_init || Tv) {
        for (int r0 = 0; r0 < ny; r0 += 65535) {
            const int r1 = std::min(ny, r0 + 65535);
            if ((e = h->L->init_rows(kp, 0, r0, r1, Tv ? Tv + (size_t)r0 * nx : nullptr, st)) != cudaSuccess)
                return cuda_bail(e, "init kernel");
        }
    } else {
        const int t_rows =
            (int)std::min<size_t>({(size_t)ny, (size_t)h->lay.stage_rows * h->lay.nq, (size_t)65535});
        for (int r0 = 0; r0 < ny; r0 += t_rows) {
            const int r1 = std::min(ny, r0 + t_rows);
            if ((e = cudaMemcpyAsync(h->stage(), p->T_init + (size_t)r0 * nx, (size_t)(r1 - r0) * nx * sizeof(double),
                                     cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_bail(e, "upload T_init");
            if ((e = h->L->init_rows(kp, 0, r0, r1, h->stage(), st)) != cudaSuccess)
                return cuda_bail(e, "init kernel");
        }
    }
    unsigned long long cnt[2] = {0, 0};
    if (gpu_maps && (e = cudaMemcpyAsync(cnt, counters, sizeof cnt, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_bail(e, "read map counters");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_bail(e, "init sync");
    if (gpu_maps) {
        if (cnt[0] != ~0ULL) {
            // name the first invalid cell as the host scan would: rescan its row
            uint8_t halfway[256] = {0};
            for (int k = 1; k <= p->n_walls; ++k) halfway[k] = 1;
            ScanResult r;
            const int y = (int)(cnt[0] / (unsigned long long)nx);
            if (scan_row_exact(p, halfway, y, nullptr, r) || r.err.empty()) {
                char buf[128];
                snprintf(buf, sizeof buf, "invalid flag map at cell (%d, %d)", (int)(cnt[0] % (unsigned long long)nx), y);
                r.err = buf;
            }
            return bail(LBM_EINVAL, r.err);
        }
        h->fluid = (int64_t)cnt[1];
    }
    h->cur = 0;
    *out = h;
    return LBM_OK;
}

lbm_status lbm_step(lbm_lattice *h, int64_t nsteps) {
    if (!h) return fail(nullptr, LBM_EINVAL, "lattice is NULL");
    if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps must be >= 0");
    if (h->batch) return fail(h, LBM_EINVAL, "lattice belongs to a batch: step it with lbm_batch_step");
    // Runs of kGraphShort steps or more replay captured graphs of kGraphSteps and kGraphShort
    // steps: the same kernels with the same arguments, without the launch gap between steps.
    // Direct launches serve short runs and remainders, a stream that is already being
    // captured (the steps then join the caller's graph), and the first run of a kernel
    // choice (its launch-time setup happens outside any capture).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(h->stream, &cs);
    if (ce != cudaSuccess) cudaGetLastError();  // leave no error behind for the launch checks
    const bool can_graph = !h->graph_off && ce == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    if (!can_graph || nsteps < kGraphShort) return step_direct(h, nsteps);
    if (!h->direct_done || h->graph_variant != h->kp.variant || h->graph_config != h->kp.config) {
        drop_graph(h);
        if (!h->direct_done) {
            lbm_status st = step_direct(h, 1);
            if (st != LBM_OK) return st;
            --nsteps;
        }
        capture_graph(h);
        if (!h->graph) return step_direct(h, nsteps);
    }
    if (h->cur != 0) {  // the graph starts from buffer 0
        lbm_status st = step_direct(h, 1);
        if (st != LBM_OK) return st;
        --nsteps;
    }
    for (; nsteps >= kGraphSteps; nsteps -= kGraphSteps) {
        cudaError_t e = cudaGraphLaunch(h->graph, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step graph");
        h->steps += kGraphSteps;
    }
    for (; nsteps >= kGraphShort; nsteps -= kGraphShort) {
        cudaError_t e = cudaGraphLaunch(h->graph_short, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step graph");
        h->steps += kGraphShort;
    }
    return step_direct(h, nsteps);
}

lbm_status lbm_sync(lbm_lattice *h) {
    if (!h) return fail(nullptr, LBM_EINVAL, "lattice is NULL");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "stream sync");
    LBM_STATUS(h);
    return LBM_OK;
}

int32_t lbm_step_kernel_count(int32_t storage, int32_t variant) {
    if (storage < LBM_F64 || storage > LBM_F16_SHIFTED) return 0;
    if (variant == LBM_STEP_AUTO || variant == LBM_STEP_SCALAR) return 1;
    if (storage == LBM_F64) return 0;
    if (variant == LBM_STEP_VEC4 || variant == LBM_STEP_VEC4W) return 5;
    if (variant == LBM_STEP_TMA) return nomrt::kTmaConfigCount;
    if (variant == LBM_STEP_VEC8) return storage == LBM_F16_SHIFTED ? 2 : 0;
    return 0;
}

lbm_status lbm_set_step_kernel(lbm_lattice *h, int32_t variant, int32_t config) {
    if (!h) return fail(nullptr, LBM_EINVAL, "lattice is NULL");
    const int32_t n = lbm_step_kernel_count(h->storage, variant);
    if (n == 0) return fail(h, LBM_EINVAL, "step variant not available for this storage");
    if (config < 0 || config >= n) return fail(h, LBM_EINVAL, "step kernel config out of range");
    if ((h->kp.tq == 9 || h->kp.bgk) && (variant == LBM_STEP_TMA || variant == LBM_STEP_VEC8))
        return fail(h, LBM_EINVAL, "the D2Q9 temperature model and BGK have the SCALAR and VEC4 step kernels only");
    if (h->kp.variant != variant || h->kp.config != config) h->direct_done = false;
    h->kp.variant = variant;
    h->kp.config = config;
    return LBM_OK;
}

lbm_status lbm_read_macro_rows(lbm_lattice *h, int32_t y0, int32_t y1, double *rho, double *ux, double *uy,
                               double *T) {
    if (!h) return fail(nullptr, LBM_EINVAL, "lattice is NULL");
    if (y0 < 0 || y1 > h->ny || y0 > y1) return fail(h, LBM_EINVAL, "rows must satisfy 0 <= y0 <= y1 <= ny");
    double *outs[4] = {rho, ux, uy, T};
    const int nx = h->nx;
    // page-locked (or device) outputs are written by the kernel in place; any pageable one sends
    // every output through the staging area
    double *direct[4] = {nullptr, nullptr, nullptr, nullptr};
    bool in_place = true;
    for (int k = 0; k < 4; ++k)
        if (outs[k]) {
            direct[k] = static_cast<double *>(const_cast<void *>(device_view(outs[k])));
            in_place = in_place && direct[k];
        }
    if (in_place) {
        for (int r0 = y0; r0 < y1; r0 += 65535) {  // the grid's y extent is at most 65535 rows per launch
            const int r1 = std::min(y1, r0 + 65535);
            double *o[4];
            for (int k = 0; k < 4; ++k) o[k] = direct[k] ? direct[k] + (size_t)(r0 - y0) * nx : nullptr;
            LBM_CUDA(h, h->L->macro_rows(h->kp, h->cur, r0, r1, o, h->stream), "macro kernel");
        }
    } else {
        const int rows = std::max(1, h->lay.stage_rows * h->lay.nq / 4);
        for (int r0 = y0; r0 < y1; r0 += rows) {
            const int r1 = std::min(y1, r0 + rows);
            const size_t n = (size_t)(r1 - r0) * nx;
            // the next chunk's kernel, queued behind these copies on the same stream, cannot
            // overwrite the staging area before they finish: one wait at the end suffices
            double *o[4];
            for (int k = 0; k < 4; ++k) o[k] = outs[k] ? h->stage() + k * n : nullptr;
            LBM_CUDA(h, h->L->macro_rows(h->kp, h->cur, r0, r1, o, h->stream), "macro kernel");
            for (int k = 0; k < 4; ++k)
                if (outs[k])
                    LBM_CUDA(h,
                             cudaMemcpyAsync(outs[k] + (size_t)(r0 - y0) * nx, h->stage() + k * n, n * sizeof(double),
                                             cudaMemcpyDeviceToHost, h->stream),
                             "read macro");
        }
    }
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "read macro sync");
    LBM_STATUS(h);
    return LBM_OK;
}

lbm_status lbm_read_macro(lbm_lattice *h, double *rho, double *ux, double *uy, double *T) {
    if (!h) return fail(nullptr, LBM_EINVAL, "lattice is NULL");
    return lbm_read_macro_rows(h, 0, h->ny, rho, ux, uy, T);
}

lbm_status lbm_nusselt(lbm_lattice *h, int32_t side, double L, double delta_T, double *nu_mean) {
    if (!h) return fail(nullptr, LBM_EINVAL, "lattice is NULL");
    if (!nu_mean) return fail(h, LBM_EINVAL, "nu_mean is NULL");
    if (side < 0 || side > 3) return fail(h, LBM_EINVAL, "side must be 0..3");
    if (!(std::isfinite(delta_T) && delta_T != 0.0)) return fail(h, LBM_EINVAL, "delta_T must be finite, non-zero");
    if (!(L > 0.0)) {
        // fluid cells across the lattice along the wall normal, on the middle line
        L = (double)(side < 2 ? h->across_x : h->across_y);
    }
    LBM_CUDA(h, h->L->nusselt(h->kp, h->cur, side, L, delta_T, h->partials(), h->stream), "nusselt kernel");
    LBM_CUDA(h, nomrt::reduce_partials(h->partials(), 2, h->result(), h->stream), "reduce kernel");
    double r[2];
    LBM_CUDA(h, cudaMemcpyAsync(r, h->result(), sizeof r, cudaMemcpyDeviceToHost, h->stream), "read nusselt");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "nusselt sync");
    LBM_STATUS(h);
    if (r[1] <= 0.0) return fail(h, LBM_EINVAL, "no fixed-temperature wall line on that side");
    *nu_mean = r[0] / r[1];
    return LBM_OK;
}

lbm_status lbm_residual(lbm_lattice *h, double *r) {
    if (!h) return fail(nullptr, LBM_EINVAL, "lattice is NULL");
    if (!r) return fail(h, LBM_EINVAL, "r is NULL");
    const int had = h->have_snap;
    LBM_CUDA(h, h->L->residual(h->kp, h->cur, h->snap(), had, h->partials(), h->stream), "residual kernel");
    LBM_CUDA(h, nomrt::reduce_partials(h->partials(), 5, h->result(), h->stream), "reduce kernel");
    double s[5];
    LBM_CUDA(h, cudaMemcpyAsync(s, h->result(), sizeof s, cudaMemcpyDeviceToHost, h->stream), "read residual");
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "residual sync");
    LBM_STATUS(h);
    h->have_snap = 1;
    if (s[4] > 0.0 || !std::isfinite(s[0]) || !std::isfinite(s[1]) || !std::isfinite(s[2]) ||
        !std::isfinite(s[3])) {
        *r = NAN;
        return fail(h, LBM_EDIVERGED, "non-finite velocity or temperature");
    }
    if (!had) {
        *r = INFINITY;
        return LBM_OK;
    }
    const double du = std::sqrt(s[1]), dT = std::sqrt(s[3]);
    const double Ru = std::sqrt(s[0]) / std::max(du, 1e-300);
    const double RT = std::sqrt(s[2]) / std::max(dT, 1e-300);
    *r = std::max(Ru, RT);
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_lattice *h, double *f9, double *g5) {
    if (!h) return fail(nullptr, LBM_EINVAL, "lattice is NULL");
    const int nx = h->nx;
    const size_t nxy = (size_t)nx * h->ny;
    for (int r0 = 0; r0 < h->ny; r0 += h->lay.stage_rows) {
        const int r1 = std::min(h->ny, r0 + h->lay.stage_rows);
        const size_t n = (size_t)(r1 - r0) * nx;
        LBM_CUDA(h, h->L->export_rows(h->kp, h->cur, r0, r1, h->stage(), h->stream), "export kernel");
        for (int q = 0; q < h->lay.nq; ++q) {
            double *dst = q < 9 ? (f9 ? f9 + q * nxy : nullptr) : (g5 ? g5 + (q - 9) * nxy : nullptr);
            if (dst)
                LBM_CUDA(h,
                         cudaMemcpyAsync(dst + (size_t)r0 * nx, h->stage() + q * n, n * sizeof(double),
                                         cudaMemcpyDeviceToHost, h->stream),
                         "export copy");
        }
    }
    // stream order keeps each chunk's kernel behind the previous chunk's copies
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "export sync");
    LBM_STATUS(h);
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_lattice *h, const double *f9, const double *g5) {
    if (!h) return fail(nullptr, LBM_EINVAL, "lattice is NULL");
    const int nx = h->nx;
    const size_t nxy = (size_t)nx * h->ny;
    const int which = (f9 ? 1 : 0) | (g5 ? 2 : 0);
    if (!which) return LBM_OK;
    for (int r0 = 0; r0 < h->ny; r0 += h->lay.stage_rows) {
        const int r1 = std::min(h->ny, r0 + h->lay.stage_rows);
        const size_t n = (size_t)(r1 - r0) * nx;
        for (int q = 0; q < h->lay.nq; ++q) {
            const double *src = q < 9 ? (f9 ? f9 + q * nxy : nullptr) : (g5 ? g5 + (q - 9) * nxy : nullptr);
            if (src)
                LBM_CUDA(h,
                         cudaMemcpyAsync(h->stage() + q * n, src + (size_t)r0 * nx, n * sizeof(double),
                                         cudaMemcpyHostToDevice, h->stream),
                         "import copy");
        }
        LBM_CUDA(h, h->L->import_rows(h->kp, h->cur, r0, r1, h->stage(), which, h->stream), "import kernel");
    }
    // one wait: the caller's arrays stay in use until the last copy has left them
    LBM_CUDA(h, cudaStreamSynchronize(h->stream), "import sync");
    return LBM_OK;
}

int32_t lbm_bounds_checking(void) { return nomrt::kBoundsBuild ? 1 : 0; }

lbm_status lbm_debug_bounds_limit(lbm_lattice *h, int64_t bytes) {
    if (!h) return fail(nullptr, LBM_EINVAL, "lattice is NULL");
    if (!nomrt::kBoundsBuild) return fail(h, LBM_EINVAL, "not a bounds-checking build");
    if (bytes < 0 || (uint64_t)bytes > (uint64_t)h->lay.total)
        return fail(h, LBM_EINVAL, "bytes must lie in 0..lbm_footprint_bytes");
    h->kp.blk_hi = h->mem + bytes;
    drop_graph(h);  // a captured graph holds the old range
    h->direct_done = false;
    return LBM_OK;
}

lbm_status lbm_info(const lbm_lattice *h, int64_t *fluid_cells, int32_t *pitch, int32_t *elem, int64_t *steps_done) {
    if (!h) return LBM_EINVAL;
    if (fluid_cells) *fluid_cells = h->fluid;
    if (pitch) *pitch = h->lay.pitch;
    if (elem) *elem = (int32_t)elem_bytes(h->storage);
    if (steps_done) *steps_done = h->steps;
    return LBM_OK;
}

const char *lbm_last_error(const lbm_lattice *h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

void lbm_destroy(lbm_lattice *h) {
    if (!h) return;
    if (h->batch) nomrt::batch_detach(h->batch, h);
    drop_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->owns_mem && h->mem) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->mem);
    }
    delete h;
}

}  // extern "C"
