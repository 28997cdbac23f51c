/*
 * nomrt_oracle.c -- plain, slow FP64 CPU oracle for the double-distribution
 * non-orthogonal MRT lattice Boltzmann method for incompressible thermal flow
 * (Q. Liu, Y.-L. He, D. Li, Q. Li, arXiv:1510.08224).
 *
 * TEST INFRASTRUCTURE. This file exists to check the CUDA path, and to be timed
 * as the CPU baseline. Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it. It shares no code, header, table or helper with the
 * CUDA library: the matrices below are the paper's printed tables, applied as
 * dense products, in the order the paper states the algorithm.
 *
 * Method (Sec. 2):
 *   flow   : D2Q9, f_bar = f - S/2 (Eq. 7); collision in moment space
 *            m* = m - Lambda (m - m_eq) + (I - Lambda/2) S~   (Eq. 8)
 *            with m = M f_bar (Eq. 10), M from Eq. 13, M^-1 from Eq. A1,
 *            m_eq from Eq. 16, S~ from Eq. 17, Lambda from Eq. 20;
 *            streaming f_bar_i(x + e_i, t + 1) = f_bar*_i(x, t) (Eq. 9).
 *   heat   : D2Q5, n* = n - Q (n - n_eq) (Eq. 24), n = N g (Eq. 26),
 *            n_eq from Eq. 28, Q from Eq. 29, N^-1 from Eq. A2; streaming Eq. 25.
 *            Or the D2Q9 temperature model of Eqs. 31-33: n = M g with the
 *            D2Q9 basis (reading A13), n_eq = M g_eq with g_eq of Eq. 31, Q of
 *            Eq. 32, alpha = c_s^2 (1/zeta_alpha - 1/2).
 *   BGK    : the single-rate special case (every rate of Eq. 20 equal to s_nu,
 *            every rate of Eq. 29 / Eq. 32 equal to zeta_alpha), selected by
 *            `collision` and written in velocity space: incompressible
 *            equilibrium, Guo-Zheng-Shi forcing, Eq. 30 or Eq. 31 for T.
 *   force  : F = g beta (T - T0) j + a (Eq. 4).
 *   macro  : rho = sum f_bar (Eq. 18), rho0 u = sum e f_bar + rho0 F / 2
 *            (Eq. 19 under the incompressible approximation, Sec. 2.1),
 *            T = sum g (Eq. 27).
 *
 * Readings where the paper is silent or inconsistent (identical on the CUDA side):
 *   A1  incompressible approximation: rho appears only in the isotropic terms
 *       (m0, the 2/3 rho of m3_eq, the rho/9 of m8_eq); every velocity-bearing
 *       term carries rho0 (= 1, Sec. 3): j = rho0 u, rho0 |u|^2, rho0 F.
 *   A2  S~_8 printed as (2/3) rho (ux Fy + uy Fx) in Eq. 17; M S of the
 *       velocity-space forcing gives (2/3) rho (ux Fx + uy Fy). The derived form
 *       is used; `s8_literal` selects the printed one (for an ablation test).
 *   A4  initial state: f_bar_i = w_i rho0, g_i = g_eq_i(T_init, u = 0) (Eq. 30).
 *   A5  halfway walls (the paper uses non-equilibrium extrapolation instead):
 *       flow    f_i(x) = f*_opp(i)(x) + 2 w_i rho0 (e_i . u_w) / cs^2
 *       T fixed g_i(x) = -g*_opp(i)(x) + 2 (varpi/4) T_w   (anti-bounce-back)
 *       adiab.  g_i(x) =  g*_opp(i)(x)
 *       for direction i arriving at fluid node x from solid node x - e_i; the
 *       wall parameters are those of the solid cell x - e_i. Solid cells hold
 *       zeros and are never updated.
 *   A6  "the fields after N steps": pull with the wall rules, then the
 *       macroscopics the (N+1)-th collision would use.
 *   A8  Nusselt (Eq. 39): second-order one-sided gradient at the halfway wall,
 *       dT/dn = (9 T_1/2 - T_3/2 - 8 T_w) / 3, midpoint average along the wall.
 *   A13 the D2Q9 temperature model's transformation (not printed): the D2Q9
 *       non-orthogonal basis M of Eq. 13. Its walls: anti-bounce-back with the
 *       even part of Eq. 31 at (T_w, u_w), bounce-back when adiabatic.
 *   A9  residual: max(|u - u_prev|_2 / |u|_2, |T - T_prev|_2 / |T|_2) over
 *       fluid nodes (u as a vector field), against the previous call's snapshot.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- tables -- */

/* D2Q9 velocities, Eq. 5 with c = 1: rest, 4 axis, 4 diagonal. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Weights below Eq. 22. */
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2, Sec. 2.1 */
static const double RHO0 = 1.0;      /* reference density, Sec. 3 */

/* Transformation matrix M, Eq. 13. */
static const double M9[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 1, 1, 1, 1, 2, 2, 2, 2},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 1, 1, 1, 1},
};

/* Its inverse, Eq. A1. */
static const double MINV9[9][9] = {
    {1, 0, 0, -1, 0, 0, 0, 0, 1},
    {0, 0.5, 0, 0.25, 0.25, 0, 0, -0.5, -0.5},
    {0, 0, 0.5, 0.25, -0.25, 0, -0.5, 0, -0.5},
    {0, -0.5, 0, 0.25, 0.25, 0, 0, 0.5, -0.5},
    {0, 0, -0.5, 0.25, -0.25, 0, 0.5, 0, -0.5},
    {0, 0, 0, 0, 0, 0.25, 0.25, 0.25, 0.25},
    {0, 0, 0, 0, 0, -0.25, 0.25, -0.25, 0.25},
    {0, 0, 0, 0, 0, 0.25, -0.25, -0.25, 0.25},
    {0, 0, 0, 0, 0, -0.25, -0.25, 0.25, 0.25},
};

/* D2Q5 transformation matrix N, Eq. 26. */
static const double N5[5][5] = {
    {1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0},
    {0, 0, 1, 0, -1},
    {0, 1, 1, 1, 1},
    {0, 1, -1, 1, -1},
};

/* Its inverse, Eq. A2. */
static const double NINV5[5][5] = {
    {1, 0, 0, -1, 0},
    {0, 0.5, 0, 0.25, 0.25},
    {0, 0, 0.5, 0.25, -0.25},
    {0, -0.5, 0, 0.25, 0.25},
    {0, 0, -0.5, 0.25, -0.25},
};

/* Opposite directions under Eq. 5's numbering. */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* ------------------------------------------------------------ interfaces -- */

typedef struct {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y;
    const uint8_t *flags;      /* ny*nx row-major; 0 fluid, k >= 1 solid of wall k */
    int32_t n_walls;
    const double *wall_u;      /* 2*n_walls: (ux, uy) of wall k at [2(k-1)] */
    const int32_t *wall_kind;  /* n_walls: 0 fixed temperature, 1 adiabatic */
    const double *wall_T;      /* n_walls */
    double nu, alpha;          /* viscosity, thermal diffusivity */
    double g_beta, T0;         /* buoyancy coefficient and reference T, Eq. 4 */
    double ax, ay;             /* external acceleration a, Eq. 4 */
    double s_e, s_q, s_eps;    /* kinetic rates of Eq. 20 */
    double zeta_e, zeta_nu;    /* kinetic rates of Eq. 29 */
    double varpi;              /* model parameter of Eq. 28 */
    int32_t s8_literal;        /* 1: the printed S~_8 of Eq. 17 (reading A2) */
    const double *T_init;      /* ny*nx or NULL (T0 everywhere) */
    const int32_t *wall_scheme; /* n_walls or NULL: 0 halfway (solid cells), 1 non-equilibrium extrapolation */
    int32_t thermal_q;         /* 5: D2Q5 (Sec. 2.2); 9: the D2Q9 model of Eqs. 31-33 */
    double theta;              /* the switch of Eq. 31, 0 or 1 (D2Q9 model) */
    double zeta_q, zeta_eps;   /* kinetic rates of Eq. 32 (D2Q9 model) */
    int32_t collision;         /* 0: the MRT collisions (Eq. 8, Eq. 24 or Eq. 32); 1: BGK (one rate each) */
    int32_t rho_in_u_terms;    /* 1: the alternative to reading A1 (rho, not rho0, in every term; ablation) */
    int32_t nee_uf_variant;    /* velocity of the fluid node inside the extrapolated non-equilibrium part
                                  (reading A11): 0 Eq. 19, (j + F/2) / rho0; ablations: 1 j / rho0,
                                  2 (j - F/2) / rho0 */
} orc_params;

/* Per-node collision inputs. s[9] is Lambda of Eq. 20; z is Q of Eq. 29 (its
 * first 5 entries, tq = 5) or of Eq. 32 (9 entries, tq = 9). */
typedef struct {
    double s[9];
    double z[9];
    double g_beta, T0, ax, ay, varpi;
    int32_t s8_literal;
    int32_t tq;
    double theta;
    int32_t bgk;   /* 1: single-relaxation-time collisions with omega = s[4], zeta = z[1] */
    int32_t rho_in_u; /* 1: rho instead of rho0 in the velocity-bearing terms of the flow collision */
} orc_rates;

typedef struct {
    int nx, ny, px, py;
    uint8_t *flags;
    int n_walls;
    double *wall_u, *wall_T;
    int *wall_kind;
    int *wall_scheme;
    uint8_t *nee_dir; /* per cell: 0, or i in 1..8 with the fluid node x_f = x + e_i of a boundary node */
    orc_rates r;
    double *f[2]; /* [9][ny*nx] */
    double *g[2]; /* [tq][ny*nx] */
    int tq;
    int cur;
    double *snap; /* residual snapshot [3][ny*nx], NULL until first call */
    int nthreads;
    double nee_half; /* the F/2 factor of u_f in nee_gather: 0.5 (Eq. 19), or 0 / -0.5 (ablations) */
    int store_bits;     /* ablation: 16 rounds every stored deviation to binary16 after each step; 0 none */
    double store_scale; /* the deviation is multiplied by this before the rounding and divided after */
} orc_lattice;

/* ------------------------------------------------------------- collision -- */

/* The flow collision of Sec. 2.1 at one node, followed by the heat collision of
 * Sec. 2.2. fbar and g are the post-streaming populations; the outputs are the
 * post-collision populations and (rho, ux, uy, T). */
void orc_collide_node(const orc_rates *r, const double fbar[9], const double g[9],
                      double fstar[9], double gstar[9], double macro[4]) {
    const int tq = r->tq == 9 ? 9 : 5;
    /* Eq. 27: temperature (the sum over the thermal lattice). */
    double T = 0.0;
    for (int i = 0; i < tq; ++i) T += g[i];
    /* Eq. 4: Boussinesq buoyancy plus the external acceleration. */
    double Fx = r->ax;
    double Fy = r->ay + r->g_beta * (T - r->T0);
    /* Eq. 18: density. */
    double rho = 0.0;
    for (int i = 0; i < 9; ++i) rho += fbar[i];
    /* Eq. 19 with j = rho0 u (incompressible approximation, reading A1); the
     * ablation rho_in_u keeps rho there and in every term below, as Eqs. 16,
     * 17 and 19 are printed. */
    const double R0 = r->rho_in_u ? rho : RHO0;
    double jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        jx += EX[i] * fbar[i];
        jy += EY[i] * fbar[i];
    }
    double ux = (jx + 0.5 * R0 * Fx) / R0;
    double uy = (jy + 0.5 * R0 * Fy) / R0;
    double uu = ux * ux + uy * uy;
    if (macro) {
        macro[0] = rho;
        macro[1] = ux;
        macro[2] = uy;
        macro[3] = T;
    }

    if (r->bgk) {
        /* BGK, the single-rate special case, written in velocity space: the
         * flow relaxes to the incompressible equilibrium (reading A1) at
         * omega = s_nu and takes the forcing term of Guo, Zheng and Shi
         * (Phys. Rev. E 65, 046308, 2002),
         *   F_i = w_i rho0 [(e_i - u) / c_s^2 + (e_i . u) e_i / c_s^4] . F,
         * weighted by 1 - omega/2; the temperature relaxes to the equilibrium
         * of Eq. 30 (D2Q5) or Eq. 31 (D2Q9) at zeta_alpha. */
        const double om = r->s[4], zt = r->z[1];
        for (int i = 0; i < 9; ++i) {
            double eu = EX[i] * ux + EY[i] * uy;
            double eF = EX[i] * Fx + EY[i] * Fy;
            double feq = W9[i] * (rho + R0 * (eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)));
            double Fi = W9[i] * R0 * (((EX[i] - ux) * Fx + (EY[i] - uy) * Fy) / CS2 + eu * eF / (CS2 * CS2));
            fstar[i] = fbar[i] - om * (fbar[i] - feq) + (1.0 - 0.5 * om) * Fi;
        }
        for (int i = 0; i < tq; ++i) {
            double eu = EX[i] * ux + EY[i] * uy;
            double geq;
            if (tq == 9)
                geq = W9[i] * T * (1.0 + eu / CS2 + r->theta * (eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)));
            else
                geq = i == 0 ? (1.0 - r->varpi) * T : 0.25 * r->varpi * T + 0.5 * eu * T;
            gstar[i] = g[i] - zt * (g[i] - geq);
        }
        return;
    }

    /* Eq. 10: m_bar = M f_bar. */
    double m[9];
    for (int k = 0; k < 9; ++k) {
        m[k] = 0.0;
        for (int i = 0; i < 9; ++i) m[k] += M9[k][i] * fbar[i];
    }
    /* Eq. 16 under reading A1. */
    double meq[9];
    meq[0] = rho;
    meq[1] = R0 * ux;
    meq[2] = R0 * uy;
    meq[3] = 2.0 / 3.0 * rho + R0 * uu;
    meq[4] = R0 * (ux * ux - uy * uy);
    meq[5] = R0 * ux * uy;
    meq[6] = 1.0 / 3.0 * R0 * uy;
    meq[7] = 1.0 / 3.0 * R0 * ux;
    meq[8] = 1.0 / 9.0 * rho + 1.0 / 3.0 * R0 * uu;
    /* Eq. 17 under readings A1 and A2. */
    double S[9];
    S[0] = 0.0;
    S[1] = R0 * Fx;
    S[2] = R0 * Fy;
    S[3] = 2.0 * R0 * (ux * Fx + uy * Fy);
    S[4] = 2.0 * R0 * (ux * Fx - uy * Fy);
    S[5] = R0 * (ux * Fy + uy * Fx);
    S[6] = 1.0 / 3.0 * R0 * Fy;
    S[7] = 1.0 / 3.0 * R0 * Fx;
    S[8] = r->s8_literal ? 2.0 / 3.0 * R0 * (ux * Fy + uy * Fx)
                         : 2.0 / 3.0 * R0 * (ux * Fx + uy * Fy);
    /* Eq. 8 with the diagonal Lambda of Eq. 20 (delta_t = 1). */
    double ms[9];
    for (int k = 0; k < 9; ++k)
        ms[k] = m[k] - r->s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * r->s[k]) * S[k];
    /* f_bar* = M^-1 m_bar* (Eq. A1). */
    for (int i = 0; i < 9; ++i) {
        fstar[i] = 0.0;
        for (int k = 0; k < 9; ++k) fstar[i] += MINV9[i][k] * ms[k];
    }

    if (tq == 9) {
        /* D2Q9 temperature model: g_eq of Eq. 31, n = M g and n_eq = M g_eq
         * (reading A13), n* = n - Q (n - n_eq) with Q of Eq. 32, g* = M^-1 n*. */
        double geq[9], n[9], neq[9], ns[9];
        for (int i = 0; i < 9; ++i) {
            double eu = EX[i] * ux + EY[i] * uy;
            geq[i] = W9[i] * T * (1.0 + eu / CS2 + r->theta * (eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)));
        }
        for (int k = 0; k < 9; ++k) {
            n[k] = 0.0;
            neq[k] = 0.0;
            for (int i = 0; i < 9; ++i) {
                n[k] += M9[k][i] * g[i];
                neq[k] += M9[k][i] * geq[i];
            }
        }
        for (int k = 0; k < 9; ++k) ns[k] = n[k] - r->z[k] * (n[k] - neq[k]);
        for (int i = 0; i < 9; ++i) {
            gstar[i] = 0.0;
            for (int k = 0; k < 9; ++k) gstar[i] += MINV9[i][k] * ns[k];
        }
    } else {
        /* Eq. 26: n = N g. */
        double n[5];
        for (int k = 0; k < 5; ++k) {
            n[k] = 0.0;
            for (int i = 0; i < 5; ++i) n[k] += N5[k][i] * g[i];
        }
        /* Eq. 28. */
        double neq[5] = {T, ux * T, uy * T, r->varpi * T, 0.0};
        /* Eq. 24 with Q of Eq. 29. */
        double ns[5];
        for (int k = 0; k < 5; ++k) ns[k] = n[k] - r->z[k] * (n[k] - neq[k]);
        /* g* = N^-1 n* (Eq. A2). */
        for (int i = 0; i < 5; ++i) {
            gstar[i] = 0.0;
            for (int k = 0; k < 5; ++k) gstar[i] += NINV5[i][k] * ns[k];
        }
    }
}

/* Fill the rate vectors from the transport coefficients:
 * nu = cs^2 (1/s_nu - 1/2) (Sec. 2.1), alpha = cs_T^2 (1/zeta_alpha - 1/2) with
 * cs_T^2 = varpi / 2 (Sec. 2.2) or cs^2 for the D2Q9 model (Eq. 33 text).
 * s0 = s1 = s2 = 1 and zeta0 = 1 as in Eqs. 20, 29, 32. */
void orc_rates_from_params(const orc_params *p, orc_rates *r) {
    double s_nu = 1.0 / (0.5 + p->nu / CS2);
    double s[9] = {1.0, 1.0, 1.0, p->s_e, s_nu, s_nu, p->s_q, p->s_q, p->s_eps};
    memcpy(r->s, s, sizeof s);
    r->tq = p->thermal_q == 9 ? 9 : 5;
    r->theta = p->theta;
    r->bgk = p->collision == 1;
    r->rho_in_u = p->rho_in_u_terms != 0;
    if (r->tq == 9) {
        /* Eq. 32 with alpha = c_s^2 (1/zeta_alpha - 1/2) */
        double z_alpha = 1.0 / (0.5 + p->alpha / CS2);
        double z[9] = {1.0, z_alpha, z_alpha, p->zeta_e, p->zeta_nu, p->zeta_nu, p->zeta_q, p->zeta_q, p->zeta_eps};
        memcpy(r->z, z, sizeof z);
    } else {
        /* Eq. 29 with alpha = c_sT^2 (1/zeta_alpha - 1/2), c_sT^2 = varpi/2 */
        double csT2 = 0.5 * p->varpi;
        double z_alpha = 1.0 / (0.5 + p->alpha / csT2);
        double z[9] = {1.0, z_alpha, z_alpha, p->zeta_e, p->zeta_nu, 0, 0, 0, 0};
        memcpy(r->z, z, sizeof z);
    }
    r->g_beta = p->g_beta;
    r->T0 = p->T0;
    r->ax = p->ax;
    r->ay = p->ay;
    r->varpi = p->varpi;
    r->s8_literal = p->s8_literal;
}

/* -------------------------------------------------------------- lattice -- */

static int wrap(int v, int n, int periodic) {
    if (!periodic) return v;
    if (v < 0) return v + n;
    if (v >= n) return v - n;
    return v;
}

/* A cell is updated every step if it is fluid or a boundary node of a wall
 * treated by non-equilibrium extrapolation; the cells of halfway walls are
 * solid and never updated. */
static int is_solid(const orc_lattice *L, int c) {
    int k = L->flags[c];
    return k != 0 && L->wall_scheme[k - 1] == 0;
}

static int is_nee(const orc_lattice *L, int c) {
    int k = L->flags[c];
    return k != 0 && L->wall_scheme[k - 1] == 1;
}

/* Post-streaming populations at fluid node (x, y), pulled from the
 * post-collision state (fsrc, gsrc) by Eqs. 9 and 25, with the wall rules of
 * reading A5 on links whose source cell is solid. */
static void gather(const orc_lattice *L, const double *fsrc, const double *gsrc, int x, int y,
                   double fin[9], double gin[9]) {
    const int nxy = L->nx * L->ny;
    const int self = y * L->nx + x;
    for (int i = 0; i < 9; ++i) {
        int sx = wrap(x - EX[i], L->nx, L->px);
        int sy = wrap(y - EY[i], L->ny, L->py);
        int src = sy * L->nx + sx;
        int k = is_solid(L, src) ? L->flags[src] : 0;
        if (k == 0) {
            fin[i] = fsrc[i * nxy + src];
        } else {
            double uwx = L->wall_u[2 * (k - 1)], uwy = L->wall_u[2 * (k - 1) + 1];
            fin[i] = fsrc[OPP[i] * nxy + self] + 2.0 * W9[i] * RHO0 * (EX[i] * uwx + EY[i] * uwy) / CS2;
        }
        if (i < L->tq) {
            if (k == 0) {
                gin[i] = gsrc[i * nxy + src];
            } else if (L->wall_kind[k - 1] == 0) {
                /* anti-bounce-back with the even part of the equilibrium at the wall:
                 * (varpi/4) T_w for Eq. 30; w_i T_w [1 + theta((e.u)^2/(2cs^4) - u^2/(2cs^2))] for Eq. 31 */
                double even;
                if (L->tq == 9) {
                    double uwx = L->wall_u[2 * (k - 1)], uwy = L->wall_u[2 * (k - 1) + 1];
                    double eu = EX[i] * uwx + EY[i] * uwy;
                    even = W9[i] * L->wall_T[k - 1] *
                           (1.0 + L->r.theta * (eu * eu / (2.0 * CS2 * CS2) - (uwx * uwx + uwy * uwy) / (2.0 * CS2)));
                } else {
                    even = (L->r.varpi / 4.0) * L->wall_T[k - 1];
                }
                gin[i] = -gsrc[OPP[i] * nxy + self] + 2.0 * even;
            } else {
                gin[i] = gsrc[OPP[i] * nxy + self];
            }
        }
    }
}

/* Incompressible equilibrium (Eq. 22 under reading A1) and the D2Q5
 * temperature equilibrium (Eq. 30) of direction i. */
static double feq_i(int i, double rho, double ux, double uy) {
    double eu = EX[i] * ux + EY[i] * uy;
    return W9[i] * (rho + RHO0 * (eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - (ux * ux + uy * uy) / (2.0 * CS2)));
}

static double geq_i(const orc_lattice *L, int i, double T, double ux, double uy) {
    if (L->tq == 9) { /* Eq. 31 */
        double eu = EX[i] * ux + EY[i] * uy;
        return W9[i] * T * (1.0 + eu / CS2 + L->r.theta * (eu * eu / (2.0 * CS2 * CS2) - (ux * ux + uy * uy) / (2.0 * CS2)));
    }
    if (i == 0) return (1.0 - L->r.varpi) * T; /* Eq. 30 */
    return 0.25 * L->r.varpi * T + 0.5 * (EX[i] * ux + EY[i] * uy) * T;
}

/* Non-equilibrium extrapolation (Z. Guo, C. Zheng, B. Shi, Chin. Phys. 11 (2002)
 * 366), the paper's default wall treatment (Sec. 3): at boundary node x_b of a
 * node-based wall, every population is the equilibrium at the wall state plus
 * the non-equilibrium part at the nearest fluid node x_f, both after streaming:
 *   f_b = f_eq(rho_f, u_w) + [f(x_f) - f_eq(rho_f, u_f)]
 *   g_b = g_eq(T_b, u_w)   + [g(x_f) - g_eq(T_f, u_f)]
 * with rho_b = rho_f, T_b = T_w for a fixed temperature and T_b = T_f for an
 * adiabatic wall; rho_f, u_f, T_f by Eqs. 18, 19, 27 with the force of Eq. 4. */
static void nee_gather(const orc_lattice *L, const double *fsrc, const double *gsrc, int x, int y,
                       double fin[9], double gin[9]) {
    int c = y * L->nx + x;
    int d = L->nee_dir[c];
    int xf = wrap(x + EX[d], L->nx, L->px), yf = wrap(y + EY[d], L->ny, L->py);
    double ff[9], gf[9];
    gather(L, fsrc, gsrc, xf, yf, ff, gf);
    double rho = 0.0, T = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += ff[i];
        jx += EX[i] * ff[i];
        jy += EY[i] * ff[i];
    }
    for (int i = 0; i < L->tq; ++i) T += gf[i];
    double Fx = L->r.ax, Fy = L->r.ay + L->r.g_beta * (T - L->r.T0);
    double ux = (jx + L->nee_half * RHO0 * Fx) / RHO0, uy = (jy + L->nee_half * RHO0 * Fy) / RHO0;
    int k = L->flags[c];
    double uwx = L->wall_u[2 * (k - 1)], uwy = L->wall_u[2 * (k - 1) + 1];
    double Tb = L->wall_kind[k - 1] == 0 ? L->wall_T[k - 1] : T;
    for (int i = 0; i < 9; ++i) fin[i] = feq_i(i, rho, uwx, uwy) + (ff[i] - feq_i(i, rho, ux, uy));
    for (int i = 0; i < L->tq; ++i) gin[i] = geq_i(L, i, Tb, uwx, uwy) + (gf[i] - geq_i(L, i, T, ux, uy));
}

/* The populations an updated cell collides: pulled for fluid, extrapolated for
 * boundary nodes. */
static void pre_collision(const orc_lattice *L, const double *fsrc, const double *gsrc, int x, int y,
                          double fin[9], double gin[9]) {
    if (L->nee_dir[y * L->nx + x]) nee_gather(L, fsrc, gsrc, x, y, fin, gin);
    else gather(L, fsrc, gsrc, x, y, fin, gin);
}

void orc_destroy(orc_lattice *L);

/* Returns NULL on invalid input: a fluid node whose pull source leaves a
 * non-periodic edge, an unknown wall id, or a size below 1. */
orc_lattice *orc_create(const orc_params *p) {
    if (p->nx < 1 || p->ny < 1 || !p->flags) return NULL;
    orc_lattice *L = (orc_lattice *)calloc(1, sizeof *L);
    if (!L) return NULL;
    L->nx = p->nx;
    L->ny = p->ny;
    L->px = p->periodic_x != 0;
    L->py = p->periodic_y != 0;
    L->nthreads = 1;
    size_t nxy = (size_t)p->nx * p->ny;
    L->flags = (uint8_t *)malloc(nxy);
    memcpy(L->flags, p->flags, nxy);
    L->n_walls = p->n_walls;
    L->wall_u = (double *)calloc(2 * (size_t)(p->n_walls + 1), sizeof(double));
    L->wall_T = (double *)calloc((size_t)p->n_walls + 1, sizeof(double));
    L->wall_kind = (int *)calloc((size_t)p->n_walls + 1, sizeof(int));
    L->wall_scheme = (int *)calloc((size_t)p->n_walls + 1, sizeof(int));
    L->nee_dir = (uint8_t *)calloc(nxy, 1);
    for (int k = 0; k < p->n_walls; ++k) {
        L->wall_u[2 * k] = p->wall_u[2 * k];
        L->wall_u[2 * k + 1] = p->wall_u[2 * k + 1];
        L->wall_T[k] = p->wall_T[k];
        L->wall_kind[k] = p->wall_kind[k];
        L->wall_scheme[k] = p->wall_scheme ? p->wall_scheme[k] : 0;
    }
    orc_rates_from_params(p, &L->r);
    L->tq = L->r.tq;
    L->nee_half = p->nee_uf_variant == 1 ? 0.0 : (p->nee_uf_variant == 2 ? -0.5 : 0.5);
    for (size_t c = 0; c < nxy; ++c)
        if (L->flags[c] > p->n_walls) { orc_destroy(L); return NULL; }
    for (int y = 0; y < L->ny; ++y)
        for (int x = 0; x < L->nx; ++x) {
            int c = y * L->nx + x;
            if (L->flags[c] == 0) {
                for (int i = 1; i < 9; ++i) {
                    int sx = wrap(x - EX[i], L->nx, L->px), sy = wrap(y - EY[i], L->ny, L->py);
                    if (sx < 0 || sx >= L->nx || sy < 0 || sy >= L->ny) { orc_destroy(L); return NULL; }
                }
            } else if (is_nee(L, c)) {
                /* the nearest fluid node: an axis neighbour if there is one, else a diagonal */
                int d = 0;
                for (int i = 1; i < 9 && !d; ++i) {
                    int sx = wrap(x + EX[i], L->nx, L->px), sy = wrap(y + EY[i], L->ny, L->py);
                    if (sx < 0 || sx >= L->nx || sy < 0 || sy >= L->ny) continue;
                    if (L->flags[sy * L->nx + sx] == 0) d = i;
                }
                if (!d) { orc_destroy(L); return NULL; }
                L->nee_dir[c] = (uint8_t)d;
            }
        }
    for (int b = 0; b < 2; ++b) {
        L->f[b] = (double *)calloc(9 * nxy, sizeof(double));
        L->g[b] = (double *)calloc((size_t)L->tq * nxy, sizeof(double));
    }
    /* Reading A4: rest equilibrium, f_bar_i = w_i rho0, g_i = g_eq_i(T_init, 0) (Eqs. 22, 30). */
    for (size_t c = 0; c < nxy; ++c) {
        if (is_solid(L, (int)c)) continue;
        double T = p->T_init ? p->T_init[c] : p->T0;
        for (int i = 0; i < 9; ++i) L->f[0][i * nxy + c] = W9[i] * RHO0;
        for (int i = 0; i < L->tq; ++i) L->g[0][i * nxy + c] = geq_i(L, i, T, 0.0, 0.0);
    }
    return L;
}

void orc_destroy(orc_lattice *L) {
    if (!L) return;
    free(L->flags);
    free(L->wall_u);
    free(L->wall_T);
    free(L->wall_kind);
    free(L->wall_scheme);
    free(L->nee_dir);
    for (int b = 0; b < 2; ++b) { free(L->f[b]); free(L->g[b]); }
    free(L->snap);
    free(L);
}

void orc_set_threads(orc_lattice *L, int n) { L->nthreads = n < 1 ? 1 : n; }

/* x rounded to the nearest IEEE 754 binary16 value (1 sign, 5 exponent, 10
 * fraction bits; ties to even; subnormals below 2^-14 in steps of 2^-24;
 * magnitudes above the largest finite value 65504 become infinite). */
double orc_round_binary16(double x) {
    if (x == 0.0 || !isfinite(x)) return x;
    const double a = fabs(x);
    int e;
    frexp(a, &e);                       /* a = m 2^e, m in [0.5, 1): binade [2^(e-1), 2^e) */
    const int E = e - 1;
    const double q = E < -14 ? ldexp(1.0, -24) : ldexp(1.0, E - 10);  /* spacing of binary16 there */
    double r = nearbyint(a / q) * q;    /* a / q is exact; the default mode rounds ties to even */
    if (r > 65504.0) r = INFINITY;
    return copysign(r, x);
}

/* Ablation (not part of the method): after every step, round the stored
 * deviation of each population from the rest state (f_bar_i - w_i rho0 and
 * g_i - w^T_i T0, the quantities a 16-bit storage of the state keeps) to
 * binary16 after multiplying it by `scale` (and divide back), as a
 * 16-bit-storage solver would; bits = 0 turns it off. For measuring what the
 * storage precision alone costs, in FP64 arithmetic otherwise. */
void orc_set_storage_rounding(orc_lattice *L, int bits, double scale) {
    L->store_bits = bits == 16 ? 16 : 0;
    L->store_scale = scale > 0.0 ? scale : 1.0;
}

static double stored(const orc_lattice *L, double v, double rest) {
    if (!L->store_bits) return v;
    return rest + orc_round_binary16((v - rest) * L->store_scale) / L->store_scale;
}

/* One time step (Eqs. 8-9, 24-25) for every fluid node, pull form. */
void orc_step(orc_lattice *L, int64_t nsteps) {
    const int nxy = L->nx * L->ny;
    for (int64_t t = 0; t < nsteps; ++t) {
        const double *fs = L->f[L->cur], *gs = L->g[L->cur];
        double *fd = L->f[1 - L->cur], *gd = L->g[1 - L->cur];
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(L->nthreads)
#endif
        for (int y = 0; y < L->ny; ++y) {
            for (int x = 0; x < L->nx; ++x) {
                int c = y * L->nx + x;
                if (is_solid(L, c)) continue;
                double fin[9], gin[9], fo[9], go[9];
                pre_collision(L, fs, gs, x, y, fin, gin);
                orc_collide_node(&L->r, fin, gin, fo, go, NULL);
                for (int i = 0; i < 9; ++i) fd[i * nxy + c] = stored(L, fo[i], W9[i] * RHO0);
                for (int i = 0; i < L->tq; ++i) gd[i * nxy + c] = stored(L, go[i], geq_i(L, i, L->r.T0, 0.0, 0.0));
            }
        }
        L->cur = 1 - L->cur;
    }
}

/* Reading A6: macroscopics at every node (solid nodes give zeros; boundary
 * nodes of extrapolated walls give their reconstructed state). */
void orc_macro(const orc_lattice *L, double *rho, double *ux, double *uy, double *T) {
    const int nxy = L->nx * L->ny;
    for (int y = 0; y < L->ny; ++y)
        for (int x = 0; x < L->nx; ++x) {
            int c = y * L->nx + x;
            double mac[4] = {0, 0, 0, 0};
            if (!is_solid(L, c)) {
                double fin[9], gin[9], fo[9], go[9];
                pre_collision(L, L->f[L->cur], L->g[L->cur], x, y, fin, gin);
                orc_collide_node(&L->r, fin, gin, fo, go, mac);
            }
            if (rho) rho[c] = mac[0];
            if (ux) ux[c] = mac[1];
            if (uy) uy[c] = mac[2];
            if (T) T[c] = mac[3];
        }
    (void)nxy;
}

/* The post-collision state, layout [9][ny*nx] and [5][ny*nx]. */
void orc_get_populations(const orc_lattice *L, double *f, double *g) {
    size_t nxy = (size_t)L->nx * L->ny;
    if (f) memcpy(f, L->f[L->cur], 9 * nxy * sizeof(double));
    if (g) memcpy(g, L->g[L->cur], (size_t)L->tq * nxy * sizeof(double));
}

void orc_set_populations(orc_lattice *L, const double *f, const double *g) {
    size_t nxy = (size_t)L->nx * L->ny;
    if (f) memcpy(L->f[L->cur], f, 9 * nxy * sizeof(double));
    if (g) memcpy(L->g[L->cur], g, (size_t)L->tq * nxy * sizeof(double));
    for (size_t c = 0; c < nxy; ++c)
        if (is_solid(L, (int)c)) {
            for (int i = 0; i < 9; ++i) L->f[L->cur][i * nxy + c] = 0.0;
            for (int i = 0; i < L->tq; ++i) L->g[L->cur][i * nxy + c] = 0.0;
        }
}

/* One step at a single fluid node, reading an external post-collision state
 * (fsrc [9][ny*nx], gsrc [5][ny*nx]) through this lattice's flags and walls.
 * Used to check single sampled nodes of very large lattices. gsrc: [tq][ny*nx]. Returns -1 if the
 * node is solid. */
int orc_update_node(const orc_lattice *L, const double *fsrc, const double *gsrc, int x, int y,
                    double fout[9], double gout[9]) {
    if (is_solid(L, y * L->nx + x)) return -1;
    double fin[9], gin[9];
    pre_collision(L, fsrc, gsrc, x, y, fin, gin);
    orc_collide_node(&L->r, fin, gin, fout, gout, NULL);
    return 0;
}

/* Eq. 39 with reading A8. side: 0 left (x min), 1 right, 2 bottom (y min), 3 top.
 * The wall is the frame line of wall cells on that side; the average runs over
 * the lines where the two nearest cells are fluid and the wall cell has a fixed
 * temperature. Nu = -L (dT/dx_axis) / dT where x_axis is x for the side walls
 * and y for the bottom and top. Returns NaN if no such line exists. */
double orc_nusselt(const orc_lattice *L, int side, double Lref, double dT) {
    double *T = (double *)malloc(sizeof(double) * (size_t)L->nx * L->ny);
    orc_macro(L, NULL, NULL, NULL, T);
    int along = (side < 2) ? L->ny : L->nx;
    double sum = 0.0;
    int count = 0;
    for (int s = 0; s < along; ++s) {
        int cw, c1, c2; /* wall cell, first and second fluid cells */
        if (side == 0) { cw = s * L->nx + 0; c1 = cw + 1; c2 = cw + 2; }
        else if (side == 1) { cw = s * L->nx + L->nx - 1; c1 = cw - 1; c2 = cw - 2; }
        else if (side == 2) { cw = s; c1 = cw + L->nx; c2 = cw + 2 * L->nx; }
        else { cw = (L->ny - 1) * L->nx + s; c1 = cw - L->nx; c2 = cw - 2 * L->nx; }
        int k = L->flags[cw];
        if (k == 0 || L->flags[c1] || L->flags[c2] || L->wall_kind[k - 1] != 0) continue;
        /* dT/ds, s measured from the wall into the fluid: a halfway wall sits half a
         * cell before c1 (reading A8); a node-based wall is the node cw itself, and
         * the one-sided second-order difference uses the nodes at 0, 1, 2. */
        double Tw = L->wall_T[k - 1];
        double dTds = L->wall_scheme[k - 1] == 1 ? (-3.0 * Tw + 4.0 * T[c1] - T[c2]) / 2.0
                                                 : (9.0 * T[c1] - T[c2] - 8.0 * Tw) / 3.0;
        double dTdaxis = (side == 0 || side == 2) ? dTds : -dTds;
        sum += -Lref * dTdaxis / dT;
        ++count;
    }
    free(T);
    return count ? sum / count : NAN;
}

/* Reading A9. R = max(|u - u_prev|_2 / |u|_2, |T - T_prev|_2 / |T|_2), the norms
 * taken over fluid nodes with u as a vector field. The first call stores the
 * snapshot and returns +inf. NaN anywhere gives NaN. */
double orc_residual(orc_lattice *L) {
    size_t nxy = (size_t)L->nx * L->ny;
    double *cur = (double *)malloc(3 * nxy * sizeof(double));
    orc_macro(L, NULL, cur, cur + nxy, cur + 2 * nxy);
    double R = INFINITY;
    if (L->snap) {
        double num_u = 0.0, den_u = 0.0, num_T = 0.0, den_T = 0.0;
        for (size_t c = 0; c < nxy; ++c) {
            if (L->flags[c]) continue;
            for (int q = 0; q < 2; ++q) {
                double d = cur[q * nxy + c] - L->snap[q * nxy + c];
                num_u += d * d;
                den_u += cur[q * nxy + c] * cur[q * nxy + c];
            }
            double d = cur[2 * nxy + c] - L->snap[2 * nxy + c];
            num_T += d * d;
            den_T += cur[2 * nxy + c] * cur[2 * nxy + c];
        }
        double du = sqrt(den_u), dT = sqrt(den_T);
        double Ru = sqrt(num_u) / (du > 1e-300 ? du : 1e-300);
        double RT = sqrt(num_T) / (dT > 1e-300 ? dT : 1e-300);
        R = (Ru != Ru || RT != RT) ? NAN : (Ru > RT ? Ru : RT);
        free(L->snap);
    }
    L->snap = cur;
    return R;
}

/* Table export for the tests that pin the oracle to the paper. */
void orc_tables(double *M, double *Minv, double *N, double *Ninv, int *ex, int *ey, double *w) {
    if (M) memcpy(M, M9, sizeof M9);
    if (Minv) memcpy(Minv, MINV9, sizeof MINV9);
    if (N) memcpy(N, N5, sizeof N5);
    if (Ninv) memcpy(Ninv, NINV5, sizeof NINV5);
    if (ex) memcpy(ex, EX, sizeof EX);
    if (ey) memcpy(ey, EY, sizeof EY);
    if (w) memcpy(w, W9, sizeof W9);
}

void orc_get_rates(const orc_lattice *L, orc_rates *r) { *r = L->r; }

int orc_threads_available(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_thermal_q(const orc_lattice *L) { return L->tq; }
