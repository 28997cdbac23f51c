/*
 * nomrt_lbm.h -- C ABI of the GB300 solver for the double-distribution
 * non-orthogonal multiple-relaxation-time lattice Boltzmann method for
 * incompressible thermal flow (Q. Liu, Y.-L. He, D. Li, Q. Li, arXiv:1510.08224).
 *
 * One call of lbm_step advances, at every fluid node, the D2Q9 flow populations
 * f_bar (Eqs. 7-9: pull streaming, raw-moment map with the non-orthogonal M of
 * Eq. 13, relaxation Eq. 8 with Eqs. 16, 17, 20, back map with M^-1 of Eq. A1)
 * and the D2Q5 temperature populations g (Eqs. 24-29, N^-1 of Eq. A2), with the
 * Boussinesq force of Eq. 4, in one fused CUDA kernel. Options: the D2Q9
 * temperature model of Eqs. 31-33 instead of D2Q5, and the single-rate (BGK)
 * special case of both collisions.
 *
 * Conventions common to every call:
 *  - Every call returns an lbm_status and never throws or aborts.
 *  - Pointers passed in are borrowed; inputs are copied before the call returns.
 *  - A lattice is bound to one CUDA stream; its calls are not thread-safe.
 *    Different lattices are independent.
 *  - Host arrays are row-major [ny][nx] planes (x fastest); population exports
 *    are [9][ny][nx] (f, directions of Eq. 5) and [5][ny][nx] (g; [9][ny][nx]
 *    with the D2Q9 temperature model).
 *  - Lengths are lattice units (delta_x = delta_t = 1, c = 1, rho0 = 1: Sec. 3).
 *  - Walls are half-way between a fluid cell and a solid cell (halfway
 *    bounce-back), or on boundary nodes (non-equilibrium extrapolation), per
 *    wall. A fluid cell at a non-periodic edge is an error: the flag map must
 *    carry a frame of wall cells there.
 */
#ifndef NOMRT_LBM_H
#define NOMRT_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,    /* invalid argument; lbm_last_error says which */
    LBM_ENOMEM = 2,    /* device allocation failed or caller block too small */
    LBM_ECUDA = 3,     /* a CUDA runtime call or launch failed */
    LBM_EDIVERGED = 4, /* NaN/Inf found in the fields (unstable run) */
    LBM_ETIMEOUT = 5   /* a kernel gave up one of its bounded waits */
} lbm_status;

/* Population storage. The FP32/FP16 forms store deviations from the rest state,
 * f_bar_i - w_i rho0 and g_i - w^T_i T0 (w^T = (1 - varpi, varpi/4 x4) for
 * D2Q5, w^T = w of the D2Q9 lattice for the model of Eqs. 31-33), and
 * compute moments and collision in FP32. LBM_F64 stores f_bar and g as they are
 * and computes in FP64. */
typedef enum { LBM_F64 = 0, LBM_F32_SHIFTED = 1, LBM_F16_SHIFTED = 2 } lbm_storage;

typedef enum { LBM_T_DIRICHLET = 0, LBM_T_ADIABATIC = 1 } lbm_thermal_kind;

typedef enum { LBM_SIDE_LEFT = 0, LBM_SIDE_RIGHT = 1, LBM_SIDE_BOTTOM = 2, LBM_SIDE_TOP = 3 } lbm_side;

/* Wall schemes. HALFWAY: the wall lies half-way between a fluid cell and the
 * wall's cells, which are solid and never updated. NEE: the wall's cells are
 * boundary nodes on the wall itself (node-based wall, the paper's setting in
 * Sec. 3), rebuilt every step by non-equilibrium extrapolation (Z. Guo,
 * C. Zheng, B. Shi, Chin. Phys. 11 (2002) 366) and then collided like fluid. */
typedef enum { LBM_WALL_HALFWAY = 0, LBM_WALL_NEE = 1 } lbm_wall_scheme;

/* One wall. Wall id k (the flag value of its cells) is walls[k-1].
 * HALFWAY flow: bounce-back with Ladd's moving-wall term,
 *   f_i(x) = f*_opp(i)(x) + 2 w_i rho0 (e_i . u_w) / c_s^2
 * for a direction i arriving at fluid cell x from a cell of this wall;
 * u_w may be tangential (a lid) or normal (a porous wall injecting fluid).
 * HALFWAY temperature: LBM_T_DIRICHLET holds the wall at its temperature T by
 * anti-bounce-back, g_i(x) = -g*_opp(i)(x) + 2 (varpi/4) T (D2Q5; the D2Q9
 * model uses twice the even part of Eq. 31 at (T, u_w));
 * LBM_T_ADIABATIC is a zero-flux wall, g_i(x) = g*_opp(i)(x).
 * NEE: at boundary node x_b with nearest fluid node x_f (an axis neighbour if
 * one is fluid, else a diagonal one), after streaming,
 *   f_b = f_eq(rho_f, u_w) + [f(x_f) - f_eq(rho_f, u_f)]
 *   g_b = g_eq(T_b, u_w) + [g(x_f) - g_eq(T_f, u_f)]
 * with T_b = T for LBM_T_DIRICHLET and T_b = T_f for LBM_T_ADIABATIC. */
typedef struct {
    double ux, uy;
    int32_t kind;   /* lbm_thermal_kind */
    int32_t scheme; /* lbm_wall_scheme */
    double T;
} lbm_wall;

/* Collision operator. MRT: Eq. 8 for the flow, Eq. 24 (or the D2Q9 model's
 * Eq. 32) for temperature. BGK: the special case with one rate each, computed in
 * velocity space,
 *   f*_i = f_i - s_nu (f_i - f_eq_i) + (1 - s_nu/2) w_i [3 (e_i - u).F + 9 (e_i.u)(e_i.F)]
 *   g*_i = g_i - zeta_alpha (g_i - g_eq_i)
 * with the incompressible f_eq (rho0 = 1), the forcing of Guo, Zheng and Shi
 * (Phys. Rev. E 65, 046308, 2002), and g_eq of Eq. 30 or Eq. 31; s_e, s_q,
 * s_eps, zeta_e, zeta_nu, zeta_q and zeta_eps are then unused (but still
 * validated). BGK lattices have the SCALAR and VEC4 step kernels only and do not
 * join fused batches. */
typedef enum { LBM_COLLISION_MRT = 0, LBM_COLLISION_BGK = 1 } lbm_collision;

/* Problem statement (Sec. 2, Eqs. 1-4) and the model's rates. */
typedef struct {
    int32_t nx, ny;               /* cells, frame included, x fastest */
    int32_t periodic_x, periodic_y;
    const uint8_t *flags;         /* ny*nx: 0 fluid, k >= 1 solid cell of wall k */
    const lbm_wall *walls;        /* n_walls entries */
    int32_t n_walls;              /* 0..254 */
    int32_t storage;              /* lbm_storage */
    double nu;                    /* viscosity: s_nu = 1 / (1/2 + nu / c_s^2), Sec. 2.1 */
    double alpha;                 /* diffusivity: zeta_alpha = 1 / (1/2 + alpha / c_sT^2), c_sT^2 = varpi/2, Sec. 2.2 */
    double g_beta;                /* buoyancy: F_y = g_beta (T - T0), Eq. 4 */
    double T0;                    /* reference temperature of Eq. 4 */
    double ax, ay;                /* external acceleration a of Eq. 4 */
    double s_e, s_q, s_eps;       /* kinetic rates of Eq. 20, each in (0, 2) */
    double zeta_e, zeta_nu;       /* kinetic rates of Eq. 29, each in (0, 2) */
    double varpi;                 /* Eq. 28 parameter, in (0, 1); the paper uses 1/2 */
    const double *T_init;         /* optional ny*nx initial temperature; NULL = T0 */
    /* Temperature lattice. 0 or 5: D2Q5 (Sec. 2.2, Eqs. 24-30). 9: the D2Q9
     * model of Eqs. 31-33, whose moments come from M of Eq. 13, with
     *   g_eq_i = w_i T [1 + e_i.u / c_s^2 + theta ((e_i.u)^2 / (2 c_s^4) - u^2 / (2 c_s^2))],
     * zeta_alpha = 1 / (1/2 + alpha / c_s^2), c_s^2 = 1/3, and varpi unused
     * (it must still lie in (0, 1)). Its halfway Dirichlet wall is
     *   g_i(x) = -g*_opp(i)(x) + 2 w_i T [1 + theta ((e_i.u_w)^2 / (2 c_s^4) - u_w^2 / (2 c_s^2))].
     * The step variants TMA and VEC8 and fused batches take D2Q5 lattices only. */
    int32_t thermal_q;
    double theta;                 /* Eq. 31: 1 keeps the second-order terms, 0 drops them (thermal_q = 9) */
    double zeta_q, zeta_eps;      /* Eq. 32 rates of the q and epsilon moments (thermal_q = 9), in (0, 2) */
    int32_t collision;            /* lbm_collision */
} lbm_params;

typedef struct lbm_lattice lbm_lattice; /* opaque; owned by the library */

/* Device bytes lbm_create needs for these parameters (populations in two
 * buffers, flag and link maps, residual snapshot, staging and reduction
 * scratch), or 0 if the parameters are invalid (lbm_last_error(NULL) says why).
 * Admission control uses it. Rows are padded to a pitch of 128 bytes of
 * storage (nx rounded up to a multiple of 16 / 32 / 64 for FP64 / FP32 / FP16);
 * ny * pitch must stay below 2^31, so the largest FP16 lattice is about
 * 2.1e9 cells (178 GB with the residual snapshot). The scalar parameters are
 * always checked; the flag map only where the size depends on it (a lattice
 * with node-based walls, whose boundary nodes take space): lbm_create and
 * lbm_validate check every flag map. */
size_t lbm_footprint_bytes(const lbm_params *p);

/* Every check lbm_create makes, on the host, without touching a GPU: the
 * scalar parameters and the flag map (wall ids within n_walls, a solid frame
 * on non-periodic edges, every fluid cell with a fluid neighbour, every
 * boundary node of a node-based wall with a fluid neighbour). LBM_OK, or
 * LBM_EINVAL with lbm_last_error(NULL) naming the first invalid cell in
 * row-major order -- the message lbm_create gives for the same map. */
lbm_status lbm_validate(const lbm_params *p);

/* Validate p, upload flags, walls and T_init, and set the initial state
 * f_bar_i = w_i rho0, g_i = g_eq_i(T_init, u = 0) of Eqs. 22 and 30 (solid cells
 * hold zeros). Where every wall is halfway, the link map is built and the flag
 * map checked on the GPU (an invalid map is reported as lbm_validate reports
 * it); flags and T_init in page-locked (or device) memory are read in place,
 * pageable ones are copied. cuda_stream: a cudaStream_t, NULL for the legacy default stream.
 * device_mem: NULL to let the library allocate, else a caller-owned device block
 * of at least lbm_footprint_bytes(p) bytes, 256-byte aligned, that must outlive
 * the lattice. On error *out is NULL and lbm_last_error(NULL) gives the reason.
 * Synchronises the stream before returning. */
lbm_status lbm_create(const lbm_params *p, void *cuda_stream, void *device_mem, size_t device_bytes,
                      lbm_lattice **out);

/* Advance nsteps >= 0 time steps (Eqs. 8-9 and 24-25, fused, one kernel per
 * step, plus one for the boundary nodes of node-based walls). Asynchronous on the
 * lattice's stream. Runs of 4 steps or more replay CUDA graphs of 32 and of 4
 * steps, captured once per step-kernel choice (the same kernels and bits,
 * without the launch gap between steps; a step launched directly first where
 * the graphs' starting buffer needs it); shorter runs and the remainder, and
 * calls on a stream that is being captured, launch the kernels directly. */
lbm_status lbm_step(lbm_lattice *h, int64_t nsteps);

/* Wait for the lattice's stream. LBM_ETIMEOUT if a step kernel gave up one of
 * its bounded waits since the last check (the state is then undefined). */
lbm_status lbm_sync(lbm_lattice *h);

/* Step kernel variants. All compute the same arithmetic and give the same
 * bits for a given storage. AUTO picks the fastest measured on GB300: the
 * scalar kernel for FP64; VEC4 for FP32 / FP16 with config 1 / 1 (MRT, D2Q5),
 * 0 / 1 (BGK, D2Q5) or 0 / 0 (D2Q9 temperature model), except VEC4W config 1
 * for FP32 MRT D2Q5 lattices whose rows are not a multiple of 512 cells.
 * SCALAR: one cell per thread. VEC4: four cells per thread with 128-bit (FP32)
 * / 64-bit (FP16) loads and warp shuffles for the x +- 1 pulls, one 512-cell
 * row segment per 128-thread block; configs 0-4 ask for 4, 5, 6, 7 or 8
 * resident blocks per SM. VEC4W: the same with one 128-cell row segment per
 * warp (four per block), so that rows that are not a multiple of 512 cells
 * leave no warp of a block idle; the same configs. Both ask L2 to prefetch
 * their segment of the link map (and, FP16, of the population planes) 32 rows
 * ahead and, where a step's grid spans more than one wave of resident blocks,
 * launch as programmatic dependents of the previous step (a step's blocks wait
 * on the device for the previous grid). VEC8 (FP16 only): eight cells per
 * thread, one 128-bit load per plane, x +- 1 realignment by byte permutes;
 * configs 0-1 ask for 4 or 3 blocks per SM. TMA: row segments staged in shared
 * memory by bulk copies in a multi-stage pipeline; its config index selects
 * the shape (cells per thread, threads per CTA, stages). */
typedef enum {
    LBM_STEP_AUTO = 0,
    LBM_STEP_SCALAR = 1,
    LBM_STEP_VEC4 = 2,
    LBM_STEP_TMA = 3,
    LBM_STEP_VEC8 = 4,
    LBM_STEP_VEC4W = 5
} lbm_step_variant;

/* Number of configs of a variant for a storage (0 if the variant does not
 * exist for it: FP64 has only SCALAR). Host only. */
int32_t lbm_step_kernel_count(int32_t storage, int32_t variant);

/* Select the step kernel of h: a variant and a config index below
 * lbm_step_kernel_count(storage, variant). LBM_EINVAL otherwise. */
lbm_status lbm_set_step_kernel(lbm_lattice *h, int32_t variant, int32_t config);

/* Macroscopic fields into caller-owned host arrays of ny*nx doubles (any may be
 * NULL): the values the next collision would use (pull with the wall rules,
 * then rho = sum f_bar (Eq. 18), rho0 u = sum e f_bar + F/2 (Eq. 19),
 * T = sum g (Eq. 27)). Solid cells read 0. Synchronises. */
lbm_status lbm_read_macro(lbm_lattice *h, double *rho, double *ux, double *uy, double *T);

/* The same for rows y0 <= y < y1 only: caller-owned host arrays of
 * (y1 - y0)*nx doubles (any may be NULL), row y at offset (y - y0)*nx. For
 * lattices whose full fields would not fit the host. LBM_EINVAL unless
 * 0 <= y0 <= y1 <= ny. Synchronises. */
lbm_status lbm_read_macro_rows(lbm_lattice *h, int32_t y0, int32_t y1, double *rho, double *ux, double *uy,
                               double *T);

/* Mean Nusselt number on a frame wall (Eq. 39): Nu = -L (dT/dx_n) / delta_T,
 * x_n = x for LEFT/RIGHT and y for BOTTOM/TOP, with the wall gradient
 * (9 T_1/2 - T_3/2 - 8 T_w) / 3 from the two nearest fluid cells and the wall's
 * fixed temperature (HALFWAY walls), or (-3 T_w + 4 T_1 - T_2) / 2 from the
 * wall node and the next two nodes (NEE walls), averaged over the lines where
 * both cells are fluid and the frame cell is a fixed-temperature wall. L <= 0 means the number of
 * fluid cells across the lattice along x_n. FP64 reduction. Synchronises.
 * LBM_EINVAL if no such line exists. */
lbm_status lbm_nusselt(lbm_lattice *h, int32_t side, double L, double delta_T, double *nu_mean);

/* Steady-state residual R = max(|u - u'|_2 / |u|_2, |T - T'|_2 / |T|_2) over
 * fluid cells, u a vector field, against the snapshot (u', T') the previous
 * call stored; every call replaces the snapshot. The first call returns
 * +infinity. FP64 reduction. LBM_EDIVERGED (and *r = NaN) if any value is NaN
 * or infinite. Synchronises. */
lbm_status lbm_residual(lbm_lattice *h, double *r);

/* Export / import the post-collision state as FP64 f_bar [9][ny][nx] and
 * g [TQ][ny][nx] host arrays, TQ = 5 or 9 (thermal_q) (shift added back or
 * removed; solid cells read 0 and are forced to 0 on import). Either pointer
 * may be NULL. Synchronises. */
lbm_status lbm_get_populations(lbm_lattice *h, double *f9, double *g5);
lbm_status lbm_set_populations(lbm_lattice *h, const double *f9, const double *g5);

/* Sizes and layout: fluid cell count, row pitch in elements, bytes of one
 * population element, steps taken since create. Any pointer may be NULL. */
lbm_status lbm_info(const lbm_lattice *h, int64_t *fluid_cells, int32_t *pitch, int32_t *elem_bytes,
                    int64_t *steps_done);

/* Steady-state residual of two macroscopic snapshots held in caller-owned
 * device memory, computed without allocating anything. The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc (a
 * serving loop whose device memory is fully budgeted by admission control, a
 * host framework that owns the allocator, a hot path that must not enter the
 * driver's allocator). Same formula as lbm_residual:
 *   R = max(|u - u_prev|_2 / |u|_2, |T - T_prev|_2 / |T|_2)
 * over the n cells whose solid[c] is 0 (solid may be NULL: every cell counts).
 * ux, uy, T, ux_prev, uy_prev, T_prev: device arrays of n doubles; solid: device
 * array of n bytes or NULL; *r: host double written on return.
 * Scratch: the reduction's block partial sums live in a fixed file-scope device
 * array (about 164 KB, held on every GPU that loads the library until the
 * process exits); n above 16,777,216 cells is rejected with LBM_EINVAL. All
 * calls share that array: calls whose kernels overlap on the GPU race.
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it with the id of
 * the device's current CUDA context; a call made in another context of that
 * device (after cudaDeviceReset or a primary-context reset) looks it up again.
 * Runs on cuda_stream (NULL = legacy default stream) with the caller's current
 * device, copies the five sums back and synchronises that stream, so it must
 * never be called on a stream that is being captured: such a call returns
 * LBM_EINVAL without touching the stream. LBM_EDIVERGED (and *r = NaN) if a
 * value is not finite. Errors: lbm_last_error(NULL). */
lbm_status lbm_residual_fields_noalloc(const double *ux, const double *uy, const double *T, const double *ux_prev,
                                       const double *uy_prev, const double *T_prev, const uint8_t *solid,
                                       int64_t n, void *cuda_stream, double *r);

/* Index checking. A library built with -DLBM_BOUNDS (the bounds-checking
 * build, _build/libnomrt_lbm_bounds.so) tests every population, link-map,
 * flag and wall-table access of the step kernels (every variant, the
 * boundary-node pass and the batch kernels) before making it: it must lie in
 * the lattice's device block, and a vector access must be aligned to its size.
 * A refused access is skipped, never made, and the first refusal's site id is
 * recorded; the next synchronising call on the lattice (lbm_sync, the
 * read-outs, lbm_batch_sync for members) returns LBM_ECUDA naming the site.
 * lbm_bounds_checking returns 1 in that build and 0 in the normal build, whose
 * checks compile to nothing. Host only. */
int32_t lbm_bounds_checking(void);

/* Test hook of the bounds-checking build: the checks of h accept only the
 * first `bytes` bytes of its device block from now on (0 <= bytes <=
 * lbm_footprint_bytes), so accesses beyond them are refused and reported as
 * above; no access outside the block is ever made. LBM_EINVAL in the normal
 * build. */
lbm_status lbm_debug_bounds_limit(lbm_lattice *h, int64_t bytes);

/* Measurement helper with no counterpart in the paper: the current device's
 * FP64 fused multiply-add rate in instructions per second (2 flops each),
 * from a kernel of independent DFMA chains on eight 256-thread blocks per SM,
 * best of five CUDA-event timed launches on cuda_stream (NULL = legacy default
 * stream). The FP64-storage step kernel is bound by this rate (its FP64
 * instructions per cell), not by HBM. Synchronises the stream. */
lbm_status lbm_probe_fp64_rate(void *cuda_stream, double *dfma_per_s);

/* ---------------------------------------------------------------- batches --
 * Many lattices of uneven size advanced together (NEXT step of the method's
 * deployment, not in the paper: the method is the same as lbm_step's, Eqs. 8-9
 * and 24-25, and a batched lattice produces the same bits as when stepped
 * alone). Members must be FP32 or FP16 storage (one storage per batch), MRT
 * with the D2Q5 temperature lattice, and bound to the batch's stream; while
 * batched, lbm_step on a member is rejected, but every other lattice call
 * (read-outs, Nusselt, residual, populations) works and sees the batch's
 * progress. Members are gathered into launch groups of up to 64 lattices
 * whose kinetic rates (s_e, s_q, s_eps, zeta_e, zeta_nu, varpi) agree; a
 * group's descriptors travel in the launch's parameter block. The batch
 * allocates with cudaMalloc two small device words (grid barrier, status) and
 * a work table of 8 bytes per 512-cell row segment of its members (where each
 * block of the batch kernels finds its member, segment and row), regrown when
 * membership changes. */
typedef struct lbm_batch lbm_batch;

/* cuda_stream: the stream every member uses (NULL = legacy default stream). */
lbm_status lbm_batch_create(void *cuda_stream, lbm_batch **out);

/* Add / remove a member. Membership changes take effect at the next step;
 * lattices may join and leave between any two steps. lbm_destroy of a member
 * removes it first. */
lbm_status lbm_batch_add(lbm_batch *b, lbm_lattice *h);
lbm_status lbm_batch_remove(lbm_batch *b, lbm_lattice *h);

/* How a batch step runs.
 * FUSED (the default): one kernel launch per step and launch group, one
 * 128-thread block of the four-cell row code per 512-cell row segment of every
 * member (a 1-D grid over the members' segments).
 * PERSISTENT: one cooperative launch per group for steps_per_launch steps: its
 * resident blocks stride over the same row segments, with a clock-bounded grid
 * barrier between steps (LBM_ETIMEOUT from lbm_batch_sync if one expires). A
 * batch holding a lattice with node-based walls runs FUSED, whose boundary-node
 * pass goes between steps.
 * CONCURRENT: each member's own single-lattice step kernel (its
 * lbm_set_step_kernel choice, read at every lbm_batch_step: a change since the
 * batch's graph was captured captures it again), the members on separate
 * streams between a fork and a join, so their kernels run side by side. */
typedef enum { LBM_BATCH_FUSED = 0, LBM_BATCH_CONCURRENT = 1, LBM_BATCH_PERSISTENT = 2 } lbm_batch_kind;
lbm_status lbm_batch_set_kind(lbm_batch *b, int32_t kind);

/* Execution mode. steps_per_launch (>= 1): steps per launch of the PERSISTENT
 * kind (default 32). graph_steps > 0 (even): steps are replayed from a CUDA
 * graph of that many steps, captured once per membership and mode; 0 launches
 * from the host. Default 32: with both at 32, a PERSISTENT batch replays one
 * persistent launch per graph. */
lbm_status lbm_batch_set_mode(lbm_batch *b, int32_t steps_per_launch, int32_t graph_steps);

/* The kind, steps per launch and graph steps in force. Any pointer may be NULL. */
lbm_status lbm_batch_get_mode(const lbm_batch *b, int32_t *kind, int32_t *steps_per_launch, int32_t *graph_steps);

/* Kernel shape of the FUSED and PERSISTENT kinds: config 0..4 asks ptxas for
 * 4..8 resident 128-thread blocks per SM (-1: the default, 6 for FP32 and 3 for
 * FP16), one block per 512-cell row segment; config 5..9, for the FUSED kind,
 * the same occupancies with one 128-cell row segment per warp (four per
 * block), so that rows that are not a multiple of 512 cells leave no warp of a
 * block idle (the PERSISTENT kind runs config c as c - 5); rows_per_unit
 * (1..1024): consecutive row segments (512 cells each, in row order) a block
 * of the persistent kernel takes per work unit (default 1). */
lbm_status lbm_batch_set_config(lbm_batch *b, int32_t config, int32_t rows_per_unit);

/* The step kernel every member runs in the CONCURRENT kind: LBM_STEP_AUTO
 * (config 0, the default) keeps each member's own lbm_set_step_kernel choice;
 * LBM_STEP_SCALAR (config 0), LBM_STEP_VEC4 or LBM_STEP_VEC4W (config 0..4)
 * runs that kernel for every member instead (the same bits; members that run
 * side by side favour other occupancies than a lattice alone). LBM_EINVAL
 * otherwise. */
lbm_status lbm_batch_set_member_kernel(lbm_batch *b, int32_t variant, int32_t config);

/* The member kernel in force (variant, config). Either pointer may be NULL. */
lbm_status lbm_batch_get_member_kernel(const lbm_batch *b, int32_t *variant, int32_t *config);

/* Autotuner: times trial_steps (>= 2) steps of every candidate on the current
 * members -- the FUSED kernel at configs 0-9, the PERSISTENT kernel at configs
 * 0-4 with work units of one and of two row segments (steps_per_launch steps
 * per launch, 32 if it is 1), and the CONCURRENT
 * kind with the members' own kernels, with every member on VEC4 at configs
 * 0-4 and on VEC4W at configs 0-4 -- each trial recomputing the current step
 * into the other buffer, so the state is unchanged; selects the fastest (kind
 * and config, or for CONCURRENT the member kernel; the PERSISTENT kind also
 * keeps the trial's steps per launch and unit size, reported as rows_per_unit
 * by lbm_batch_info), and returns the kind in *best_kind, in
 * *best_config the config (FUSED, PERSISTENT) or, for CONCURRENT, -1 (members'
 * own), 0-4 (VEC4 config c) or 5-9 (VEC4W config c - 5), and the mean ms per
 * step of every candidate in ms_per_step[31] (FUSED 0-9, PERSISTENT 0-4 with
 * one-segment units, PERSISTENT 0-4 with two-segment units, CONCURRENT own,
 * CONCURRENT VEC4 0-4, CONCURRENT VEC4W 0-4; +inf for a
 * candidate that cannot run, such as PERSISTENT with node-based walls). Any
 * output may be NULL. Synchronises. */
lbm_status lbm_batch_tune(lbm_batch *b, int32_t trial_steps, int32_t *best_kind, int32_t *best_config,
                          float *ms_per_step);

/* Advance every member by nsteps (asynchronous on the batch's stream). */
lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps);

/* Wait for the batch's stream; LBM_ETIMEOUT if a persistent launch gave up a
 * grid barrier (the members' state is then undefined; later persistent
 * launches return at once until this call clears the status). */
lbm_status lbm_batch_sync(lbm_batch *b);

/* Test hook for the timeout path. With extra = 1 the persistent kernel's grid
 * barrier waits for one more arrival than the grid has, so its bounded wait
 * (about 2 s) expires on purpose: the kernel records the timeout in the batch's
 * status word and returns, and the next lbm_batch_sync reports LBM_ETIMEOUT
 * (the members' state is then undefined). No fault and no hang are involved.
 * extra = 0 restores normal operation. LBM_EINVAL for other values. */
lbm_status lbm_batch_debug_barrier_extra(lbm_batch *b, int32_t extra);

/* The steady-state residual of every member (lbm_residual's R, against and
 * then replacing each member's own snapshot; +infinity at a member's first
 * call), with one synchronisation for the whole batch: the members' residual
 * kernels run on the batch's stream, their sums land side by side and come
 * back in one copy. members[i] (may be NULL) and r[i] for i < *n, in the
 * batch's member order; cap: the capacity of both arrays (LBM_EINVAL if
 * below the member count, *n still set). A member whose fields are not finite
 * gets r[i] = NaN (lbm_residual would return LBM_EDIVERGED for it). The batch
 * allocates its device and pinned host buffers for the sums (cudaMalloc,
 * cudaHostAlloc) when it first needs them. Synchronises. */
lbm_status lbm_batch_residuals(lbm_batch *b, int32_t cap, lbm_lattice **members, double *r, int32_t *n);

/* Members, their fluid cells, 512-cell row segments per step (summed over the
 * launch groups), config in force (-1 for the CONCURRENT kind), rows per unit,
 * batch steps taken. Any pointer may be NULL. */
lbm_status lbm_batch_info(const lbm_batch *b, int32_t *members, int64_t *cells, int32_t *units, int32_t *config,
                          int32_t *rows_per_unit, int64_t *steps_done);

/* Last error of b (never NULL); with b == NULL, the thread's last error. */
const char *lbm_batch_last_error(const lbm_batch *b);

/* Free the batch; its members stay valid and become unbatched. */
void lbm_batch_destroy(lbm_batch *b);

/* Last error message of h (never NULL); with h == NULL, the calling thread's
 * last lbm_create / lbm_footprint_bytes / lbm_residual_fields_noalloc error. */
const char *lbm_last_error(const lbm_lattice *h);

/* Free the lattice (and its device memory if the library allocated it). */
void lbm_destroy(lbm_lattice *h);

#ifdef __cplusplus
}
#endif

#endif /* NOMRT_LBM_H */
