// Internal interface between the C-ABI host code (lbm_api.cu) and the
// per-storage kernel translation units (kernels_f64.cu, kernels_f32.cu,
// kernels_f16.cu). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <atomic>
#include <stdint.h>

namespace nomrt {

// Number of populations per node: 9 (D2Q9 flow, Eq. 5) + 5 (D2Q5 temperature);
// kQmax with the D2Q9 temperature model of Eqs. 31-33 (9 + 9).
constexpr int kQ = 14;
constexpr int kQmax = 18;
// Devices a process may use; per-device launch caches hold one slot each.
constexpr int kMaxDevices = 64;
// Link-map value of a solid cell (and of the row padding).
constexpr uint8_t kSolid = 0xFF;
// Fixed number of blocks of the reduction kernels (deterministic sums).
constexpr int kRedBlocks = 512;
constexpr int kRedThreads = 256;
// Device status word values (set by kernels, read and cleared by the host).
constexpr int kStatusOk = 0;
constexpr int kStatusTimeout = 1;
// Whether this build checks every step-kernel access against the lattice's
// device block (compiled with -DLBM_BOUNDS; see in_block in nomrt_kernels.cuh).
#ifdef LBM_BOUNDS
constexpr bool kBoundsBuild = true;
#else
constexpr bool kBoundsBuild = false;
#endif
// Step kernel variants (lbm_set_step_variant).
constexpr int kStepAuto = 0;
constexpr int kStepScalar = 1;
constexpr int kStepVec4 = 2;
constexpr int kStepTma = 3;
constexpr int kStepVec8 = 4;
constexpr int kStepVec4w = 5;
// Shapes of the TMA step kernel (see launchers.cuh).
constexpr int kTmaConfigCount = 5;

// Per-wall constants, indexed by wall id (entry 0 unused). cf[i] is Ladd's
// moving-wall term 2 w_i rho0 (e_i . u_w) / c_s^2 for direction i; a
// temperature link from the wall gives g_i = tsgn * g*_opp(i) + tb, with
// tsgn = -1, tb = (varpi/2)(T_w - T_ref) for a fixed temperature T_w
// (anti-bounce-back) and tsgn = +1, tb = 0 for an adiabatic wall.
struct WallDev {
    double cf[9];
    double tsgn;
    double tb;
    double Tw;
    double uwx, uwy;  // wall velocity
    double nee;       // 1: node-based wall (non-equilibrium extrapolation), 0: halfway
    double adiabatic; // 1: adiabatic, 0: fixed temperature
    double tb9[9];    // D2Q9 temperature model: g_i = tsgn g*_opp(i) + tb9[i]
};

// Everything a kernel needs to know about one lattice, in FP64; each kernel
// translation unit converts the rates to its compute type.
struct KParams {
    int nx, ny, pitch;
    int px, py;                 // periodic x / y
    size_t plane;               // elements per population plane (ny * pitch)
    void *pop[2];               // the two ping-pong buffers, kQ planes each
    const uint8_t *mask;        // link map: bit i-1 set if direction i pulls from a solid cell
    const uint8_t *flags;       // wall ids
    const WallDev *walls;
    // rates and constants
    double s_e, s_nu, s_q, s_eps;     // Eq. 20
    double z_a, z_e, z_nu;            // Eq. 29
    double g_beta, T0, ax, ay, varpi; // Eq. 4, Eq. 28
    double rho_ref, T_ref;            // storage shift (0 for FP64 storage)
    int tq;                           // temperature lattice: 5 (D2Q5) or 9 (Eqs. 31-33)
    double theta, z_q, z_eps;         // Eq. 31 switch, Eq. 32 rates (tq = 9)
    int bgk;                          // 1: single-rate (BGK) collisions
    const int2 *nee;                  // boundary nodes of NEE walls: (cell offset, dir | wall id << 8)
    int n_nee;
    const uint8_t *nee_dir;           // per cell: 0, or the direction i of the nearest fluid node x + e_i
    int variant;                      // step kernel variant (kStep*)
    int config;                       // shape index within the variant (TMA: 0..kTmaConfigs-1)
    int *status;                      // device status word
    // bounds-checking build (-DLBM_BOUNDS): the lattice's device block [blk_lo, blk_hi), which
    // every checked access must stay in, and the word that records the first failing check
    const char *blk_lo, *blk_hi;
    int *oob;
};

// Launchers, one set per storage type (0 = f64, 1 = f32-shifted, 2 = f16-shifted).
// All are asynchronous on `st` and return the launch error.
struct Launchers {
    // one fused stream-and-collide step reading buffer `src`, writing 1 - src
    // (boundary nodes of NEE walls included)
    cudaError_t (*step)(const KParams &, int src, cudaStream_t st);
    // the boundary nodes of NEE walls alone (after a step kernel that skipped them)
    cudaError_t (*nee)(const KParams &, int src, cudaStream_t st);
    // initial state into buffer `buf`, rows [r0, r1), zeros into the other buffer; T rows in `T`
    // (device-readable, (r1-r0)*nx), or nullptr for T0 everywhere
    cudaError_t (*init_rows)(const KParams &, int buf, int r0, int r1, const double *T, cudaStream_t st);
    // macroscopics of rows [r0, r1) into out[0..3] (rho, ux, uy, T; (r1-r0)*nx doubles each, any NULL)
    cudaError_t (*macro_rows)(const KParams &, int buf, int r0, int r1, double *const out[4], cudaStream_t st);
    // FP64 export / import of rows [r0, r1): out/in [9 + tq][(r1-r0)*nx]
    cudaError_t (*export_rows)(const KParams &, int buf, int r0, int r1, double *out, cudaStream_t st);
    cudaError_t (*import_rows)(const KParams &, int buf, int r0, int r1, const double *in, int which,
                               cudaStream_t st);
    // Nusselt partial sums (sum, count) per block into partials[kRedBlocks][2]
    cudaError_t (*nusselt)(const KParams &, int buf, int side, double L, double dT, double *partials,
                           cudaStream_t st);
    // residual partial sums (|du|^2, |u|^2, dT^2, T^2, nonfinite) per block into
    // partials[kRedBlocks][5]; updates snap[3][plane] (ux, uy, T)
    cudaError_t (*residual)(const KParams &, int buf, double *snap, int have_snap, double *partials,
                            cudaStream_t st);
};

const Launchers &launchers_f64();
const Launchers &launchers_f32();
const Launchers &launchers_f16();

// Sets the calling thread's error message (lbm_last_error(NULL)).
void set_thread_error(const char *msg);

// Final fixed-order reduction of partials[kRedBlocks][width] into out[width].
cudaError_t reduce_partials(const double *partials, int width, double *out, cudaStream_t st);

}  // namespace nomrt
