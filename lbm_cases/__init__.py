"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the
benchmark.

This module holds no arithmetic of the lattice Boltzmann method. It only lays out
problems: the flag map (0 = fluid, k >= 1 = solid cell of wall k), the wall table,
the physical parameters (viscosity, diffusivity, buoyancy coefficient) obtained
from the dimensionless groups that define each problem (Re, Pr, Ra, Ma), and the
initial temperature field drawn from a counter-based generator (SplitMix64, with
Box-Muller for Gaussian draws). Relaxation rates are derived from nu and alpha on
each side separately.

Geometry convention: walls sit half-way between the last fluid cell and a frame of
solid cells, so a problem with H fluid rows has ny = H + 2 cells on a
non-periodic y axis and the characteristic length is H.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np

DIRICHLET = 0
ADIABATIC = 1
# wall schemes: halfway walls between a fluid cell and a frame of solid cells, or
# node-based walls whose boundary nodes are reconstructed by non-equilibrium
# extrapolation (the paper's default, Sec. 3)
HALFWAY = 0
NEE = 1

# kinetic rates used for the convection problems of Sec. 3.4 of the paper
KINETIC_CONVECTION = dict(s_e=1.6, s_q=1.2, s_eps=1.8, zeta_e=1.9, zeta_nu=1.9)
# "the remaining relaxation rates are set to be 1.0" (Secs. 3.1, 3.3)
KINETIC_ONE = dict(s_e=1.0, s_q=1.0, s_eps=1.0, zeta_e=1.0, zeta_nu=1.0)

CS2 = 1.0 / 3.0  # D2Q9 lattice sound speed squared (lattice units, c = 1)


@dataclass
class Wall:
    ux: float = 0.0
    uy: float = 0.0
    kind: int = ADIABATIC
    T: float = 0.0
    scheme: int = HALFWAY


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    periodic_x: bool
    periodic_y: bool
    flags: np.ndarray               # (ny, nx) uint8
    walls: list                     # wall k = walls[k-1]
    nu: float
    alpha: float
    g_beta: float = 0.0
    T0: float = 0.0
    delta_T: float = 1.0
    ax: float = 0.0
    ay: float = 0.0
    s_e: float = 1.0
    s_q: float = 1.0
    s_eps: float = 1.0
    zeta_e: float = 1.0
    zeta_nu: float = 1.0
    varpi: float = 0.5
    T_init: np.ndarray | None = None  # (ny, nx) float64
    L: float = 1.0                  # characteristic length for Nu
    meta: dict = field(default_factory=dict)
    thermal_q: int = 5              # 5: D2Q5 temperature (Sec. 2.2); 9: the D2Q9 model (Eqs. 31-33)
    theta: float = 1.0              # the switch of Eq. 31 (D2Q9 model)
    zeta_q: float = 1.0             # kinetic rates of Eq. 32 (D2Q9 model)
    zeta_eps: float = 1.0
    collision: int = 0              # 0: the MRT collisions; 1: BGK (one rate for f, one for g)

    @property
    def fluid_nodes(self) -> int:
        return int(np.count_nonzero(self.flags == 0))

    def with_(self, **kw) -> "Case":
        return replace(self, **kw)


# ------------------------------------------------------------------ random --

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of SplitMix64 (Steele, Lea, Flood 2014) starting at counter
    `offset`: output k mixes seed + (k + 1) * 0x9E3779B97F4A7C15."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of SplitMix64 times 2^-53."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed: int, n: int) -> np.ndarray:
    """Standard normal draws by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:n]


# ---------------------------------------------------------------- geometry --

def _frame_y(nx: int, H: int, bottom: int, top: int) -> np.ndarray:
    """Periodic-x channel: fluid rows 1..H, solid rows 0 (wall `bottom`) and H+1 (`top`)."""
    flags = np.zeros((H + 2, nx), dtype=np.uint8)
    flags[0, :] = bottom
    flags[-1, :] = top
    return flags


def _frame_box(n_x: int, n_y: int, left: int, right: int, bottom: int, top: int) -> np.ndarray:
    """Closed box of n_x x n_y fluid cells inside a one-cell solid frame. The four
    corner cells take the side walls' ids (left / right)."""
    flags = np.zeros((n_y + 2, n_x + 2), dtype=np.uint8)
    flags[0, :] = bottom
    flags[-1, :] = top
    flags[:, 0] = left
    flags[:, -1] = right
    return flags


def fluid_y(H: int) -> np.ndarray:
    """Wall-normal positions of the fluid rows in units of H (halfway walls)."""
    return (np.arange(H) + 0.5) / H


# ----------------------------------------------------------------- problems --

def porous_couette(H: int = 64, nx: int = 8, Re: float = 5.0, Pr: float = 0.71, Ra: float = 100.0,
                   U0: float = 0.1, v0: float = 0.01, s_kin=(1.1, 1.2), T_h: float = 1.0,
                   T_c: float = 0.0) -> Case:
    """Thermal channel with wall injection (Sec. 3.3 of the paper): bottom plate
    static and cold, top plate moving at U0 and hot, uniform injection v0 through
    the bottom and suction through the top. Re = H v0 / nu, Pr = nu / alpha,
    Ra = g beta dT H^3 / (nu alpha). s_kin = (a, b) sets s_e = s_eps = zeta_e = a
    and s_q = zeta_nu = b."""
    nu = H * v0 / Re
    alpha = nu / Pr
    dT = T_h - T_c
    g_beta = Ra * nu * alpha / (dT * H ** 3)
    walls = [Wall(0.0, v0, DIRICHLET, T_c), Wall(U0, v0, DIRICHLET, T_h)]
    a, b = s_kin
    return Case("porous_couette", nx, H + 2, True, False, _frame_y(nx, H, 1, 2), walls,
                nu=nu, alpha=alpha, g_beta=g_beta, T0=0.5 * (T_h + T_c), delta_T=dT,
                s_e=a, s_q=b, s_eps=a, zeta_e=a, zeta_nu=b, L=float(H),
                meta=dict(Re=Re, Pr=Pr, Ra=Ra, U0=U0, v0=v0, T_h=T_h, T_c=T_c, H=H))


def porous_couette_exact(case: Case):
    """Closed-form steady profiles of the injection channel: Eq. 36 (u_x) and
    Eq. 37 (T), at the fluid-row positions."""
    m = case.meta
    y = fluid_y(m["H"])
    Re, Pr = m["Re"], m["Pr"]
    ux = m["U0"] * np.expm1(Re * y) / np.expm1(Re)
    T = m["T_c"] + (m["T_h"] - m["T_c"]) * np.expm1(Pr * Re * y) / np.expm1(Pr * Re)
    return ux, T


def couette(H: int = 16, nx: int = 4, U0: float = 0.05, nu: float = 0.1, T_bot: float = 0.0,
            T_top: float = 1.0, alpha: float = 0.05, kinetic=None) -> Case:
    """Plane Couette flow with conduction between two plates (no injection, no
    buoyancy): steady u_x and T are linear in y."""
    kin = dict(KINETIC_ONE if kinetic is None else kinetic)
    walls = [Wall(0.0, 0.0, DIRICHLET, T_bot), Wall(U0, 0.0, DIRICHLET, T_top)]
    return Case("couette", nx, H + 2, True, False, _frame_y(nx, H, 1, 2), walls, nu=nu,
                alpha=alpha, T0=0.5 * (T_bot + T_top), delta_T=T_top - T_bot, L=float(H),
                meta=dict(U0=U0, H=H, T_bot=T_bot, T_top=T_top), **kin)


def poiseuille(H: int = 30, nx: int = 4, ax: float = 2e-6, nu: float = 1.0 / 6.0, kinetic=None) -> Case:
    """Channel flow between static plates driven by a body force a = (ax, 0)
    (Sec. 3.1). Steady profile u_x = ax y (H - y) / (2 nu)."""
    kin = dict(KINETIC_ONE if kinetic is None else kinetic)
    walls = [Wall(0.0, 0.0, ADIABATIC, 0.0), Wall(0.0, 0.0, ADIABATIC, 0.0)]
    return Case("poiseuille", nx, H + 2, True, False, _frame_y(nx, H, 1, 2), walls, nu=nu,
                alpha=0.1, ax=ax, L=float(H), meta=dict(H=H, ax=ax), **kin)


def convection_params(L: float, Ra: float, Pr: float, Ma: float, dT: float = 1.0):
    """nu, alpha, g beta from the definitions Ra = g beta dT L^3 / (nu alpha),
    Pr = nu / alpha, Ma = u_c / c_s with u_c = sqrt(g beta dT L) (Sec. 3.4)."""
    u_c = Ma * math.sqrt(CS2)
    g_beta = u_c * u_c / (L * dT)
    nu = u_c * L * math.sqrt(Pr / Ra)
    return nu, nu / Pr, g_beta


def cavity(n: int = 256, Ra: float = 1e5, Pr: float = 0.71, Ma: float = 0.1, seed: int = 0,
           noise: float = 1e-6, T_h: float = 1.0, T_c: float = 0.0, n_y: int | None = None) -> Case:
    """Differentially heated square cavity (Sec. 3.4): left wall hot, right wall
    cold, top and bottom adiabatic, all no-slip. T_init = (T_h + T_c)/2 plus
    uniform noise in [-noise, noise) from SplitMix64(seed)."""
    n_y = n if n_y is None else n_y
    dT = T_h - T_c
    nu, alpha, g_beta = convection_params(float(n), Ra, Pr, Ma, dT)
    walls = [Wall(0, 0, DIRICHLET, T_h), Wall(0, 0, DIRICHLET, T_c), Wall(0, 0, ADIABATIC, 0.0),
             Wall(0, 0, ADIABATIC, 0.0)]
    flags = _frame_box(n, n_y, 1, 2, 3, 4)
    T0 = 0.5 * (T_h + T_c)
    Ti = np.zeros(flags.shape)
    fl = flags == 0
    Ti[fl] = T0 + noise * (2.0 * uniform01(seed, int(fl.sum())) - 1.0)
    return Case("cavity", n + 2, n_y + 2, False, False, flags, walls, nu=nu, alpha=alpha,
                g_beta=g_beta, T0=T0, delta_T=dT, T_init=Ti, L=float(n),
                meta=dict(Ra=Ra, Pr=Pr, Ma=Ma, seed=seed), **KINETIC_CONVECTION)


def rayleigh_benard(nx: int = 4096, H: int = 2048, Ra: float = 1e6, Pr: float = 0.71, Ma: float = 0.1,
                    seed: int = 0, sigma: float = 1e-3, T_h: float = 1.0, T_c: float = 0.0,
                    L: float | None = None) -> Case:
    """Rayleigh-Benard cell periodic in x: bottom plate hot, top plate cold,
    both no-slip. T_init = the linear conduction profile plus N(0, sigma^2)
    from SplitMix64(seed) with Box-Muller. The length scale is H unless L is
    given (a crop run at the same nu, alpha, g beta as a larger cell)."""
    Lc = float(H) if L is None else float(L)
    dT = T_h - T_c
    nu, alpha, g_beta = convection_params(Lc, Ra, Pr, Ma, dT)
    walls = [Wall(0, 0, DIRICHLET, T_h), Wall(0, 0, DIRICHLET, T_c)]
    flags = _frame_y(nx, H, 1, 2)
    Ti = np.zeros(flags.shape)
    prof = T_h - dT * fluid_y(H)
    Ti[1:-1, :] = prof[:, None]
    if sigma:
        Ti[1:-1, :] += sigma * gaussian(seed, nx * H).reshape(H, nx)
    return Case("rayleigh_benard", nx, H + 2, True, False, flags, walls, nu=nu, alpha=alpha,
                g_beta=g_beta, T0=0.5 * (T_h + T_c), delta_T=dT, T_init=Ti, L=Lc,
                meta=dict(Ra=Ra, Pr=Pr, Ma=Ma, seed=seed, sigma=sigma), **KINETIC_CONVECTION)


def periodic_box(nx: int, ny: int, nu: float = 0.05, alpha: float = 0.05, g_beta: float = 0.0,
                 T0: float = 0.0, T_init=None, kinetic=None, ax: float = 0.0, ay: float = 0.0) -> Case:
    """Fully periodic lattice with no walls."""
    kin = dict(KINETIC_ONE if kinetic is None else kinetic)
    return Case("periodic", nx, ny, True, True, np.zeros((ny, nx), np.uint8), [], nu=nu, alpha=alpha,
                g_beta=g_beta, T0=T0, T_init=T_init, ax=ax, ay=ay, L=float(ny), **kin)


def random_state(case: Case, seed: int, amp_f: float = 0.02, amp_g: float = 0.05):
    """A seeded non-equilibrium population state for parity checks: rest
    weights w_i plus uniform noise for the flow, T0 shares plus noise for the
    temperature; zeros on solid cells (cells of halfway walls). Layout
    (9, ny, nx) and (thermal_q, ny, nx)."""
    w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    tq = getattr(case, "thermal_q", 5)
    wT = w9 if tq == 9 else np.array([1 - case.varpi] + [case.varpi / 4] * 4)
    n = case.nx * case.ny
    f = w9[:, None] + amp_f * (2 * uniform01(seed, 9 * n).reshape(9, n) - 1)
    g = (case.T0 + 0.3) * wT[:, None] + amp_g * (2 * uniform01(seed + 1, tq * n).reshape(tq, n) - 1)
    flags = case.flags.reshape(-1)
    solid = np.array([k != 0 and case.walls[k - 1].scheme == HALFWAY for k in flags], dtype=bool)
    f[:, solid] = 0.0
    g[:, solid] = 0.0
    return f.reshape(9, case.ny, case.nx), g.reshape(tq, case.ny, case.nx)


def obstacle_channel(nx: int = 37, H: int = 11, frac: float = 0.12, seed: int = 1, U0: float = 0.04,
                     nu: float = 0.04, alpha: float = 0.05, g_beta: float = 1e-3) -> Case:
    """Periodic-x channel with a moving, heated lid (wall 2), a cold static
    bottom (wall 1) and randomly placed solid cells (adiabatic wall 3) drawn
    from SplitMix64(seed). Fluid cells left without a fluid neighbour are
    filled, so every fluid cell has at least one fluid neighbour."""
    flags = _frame_y(nx, H, 1, 2)
    u = uniform01(seed, nx * H).reshape(H, nx)
    inner = flags[1:-1]
    inner[u < frac] = 3
    EXY = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    ny = H + 2
    for y in range(1, ny - 1):
        for x in range(nx):
            if flags[y, x]:
                continue
            if all(flags[y - dy, (x - dx) % nx] for dx, dy in EXY):
                flags[y, x] = 3
    walls = [Wall(0, 0, DIRICHLET, 0.0), Wall(U0, 0, DIRICHLET, 1.0), Wall(0, 0, ADIABATIC, 0.0)]
    Ti = np.where(flags == 0, 0.5, 0.0)
    return Case("obstacle_channel", nx, ny, True, False, flags, walls, nu=nu, alpha=alpha, g_beta=g_beta,
                T0=0.5, T_init=Ti, L=float(H), meta=dict(seed=seed), **KINETIC_CONVECTION)


def batched_cavities(count: int = 64, side_lo: int = 128, side_hi: int = 1024, ra_lo: float = 1e3,
                     ra_hi: float = 1e6, Pr: float = 0.71, Ma: float = 0.1, seed: int = 0):
    """Differentially heated cavities of uneven size: side lengths uniform over
    the integers side_lo..side_hi and Ra log-uniform in [ra_lo, ra_hi], both
    drawn from SplitMix64(seed); each cavity's initial noise uses seed + 1 + k."""
    u = uniform01(seed, 2 * count)
    sides = side_lo + np.floor(u[0::2] * (side_hi - side_lo + 1)).astype(int)
    ras = np.exp(np.log(ra_lo) + u[1::2] * (np.log(ra_hi) - np.log(ra_lo)))
    return [cavity(n=int(n), Ra=float(ra), Pr=Pr, Ma=Ma, seed=seed + 1 + k) for k, (n, ra) in
            enumerate(zip(sides, ras))]


def serving_stream(n: int = 40, rate: float = 20.0, seed: int = 0, side_lo: int = 64, side_hi: int = 2048,
                   ra_lo: float = 1e3, ra_hi: float = 1e6, Pr: float = 0.71, Ma: float = 0.1,
                   cavity_share: float = 0.5, rb_ra=None):
    """n requests with Poisson arrivals (exponential gaps of mean 1/rate from
    SplitMix64(seed)); each is a cavity (side s) with probability
    cavity_share, else a Rayleigh-Benard cell (s x s/2, periodic in x), s
    log-uniform over [side_lo, side_hi], Ra log-uniform over [ra_lo, ra_hi]
    (for the Rayleigh-Benard cells over rb_ra = (lo, hi) instead, if given).
    Returns [(arrival seconds, kind, case)]."""
    u = uniform01(seed, 4 * n)
    gaps = -np.log(1.0 - u[0::4]) / rate
    arrivals = np.cumsum(gaps) - gaps[0]
    sides = np.exp(np.log(side_lo) + u[1::4] * (np.log(side_hi) - np.log(side_lo)))
    ras = np.exp(np.log(ra_lo) + u[2::4] * (np.log(ra_hi) - np.log(ra_lo)))
    out = []
    for k in range(n):
        s = max(8, int(round(sides[k])))
        if u[4 * k + 3] < cavity_share:
            case = cavity(n=s, Ra=float(ras[k]), Pr=Pr, Ma=Ma, seed=seed + 100 + k)
            kind = "cavity"
        else:
            ra = float(ras[k])
            if rb_ra is not None:  # the same uniform draw, mapped onto the Rayleigh-Benard range
                ra = float(np.exp(np.log(rb_ra[0]) + u[4 * k + 2] * (np.log(rb_ra[1]) - np.log(rb_ra[0]))))
            case = rayleigh_benard(nx=s, H=max(4, s // 2), Ra=ra, Pr=Pr, Ma=Ma, seed=seed + 100 + k)
            kind = "rayleigh_benard"
        out.append((float(arrivals[k]), kind, case))
    return out


# --------------------------------------------------- node-based (NEE) walls --

def node_y(H: int) -> np.ndarray:
    """Wall-normal positions of the nodes 0..H of a node-based channel, in units of H."""
    return np.arange(H + 1) / H


def poiseuille_nee(H: int = 60, nx: int = 6, ax: float = 2e-6, s_nu: float = 1.754, kinetic=None) -> Case:
    """Sec. 3.1 as the paper sets it up: walls on the nodes y = 0 and y = H
    (H + 1 rows of nodes, non-equilibrium extrapolation), periodic x, body
    force a = (ax, 0), s_nu given, the other rates 1. Exact profile (Eq. 34):
    u_x = ax y (H - y) / (2 nu)."""
    kin = dict(KINETIC_ONE if kinetic is None else kinetic)
    nu = (1.0 / s_nu - 0.5) * CS2
    walls = [Wall(0.0, 0.0, ADIABATIC, 0.0, NEE), Wall(0.0, 0.0, ADIABATIC, 0.0, NEE)]
    flags = np.zeros((H + 1, nx), np.uint8)
    flags[0, :] = 1
    flags[-1, :] = 2
    return Case("poiseuille_nee", nx, H + 1, True, False, flags, walls, nu=nu, alpha=0.1, ax=ax, L=float(H),
                meta=dict(H=H, ax=ax, nodes=True), **kin)


def porous_couette_nee(H: int = 60, nx: int = 6, Re: float = 10.0, Pr: float = 0.71, U0: float = 0.01,
                       v0: float = 0.01, s_nu: float | None = None, T_h: float = 1.0, T_c: float = 0.0) -> Case:
    """Sec. 3.3 as the paper sets it up: node-based walls at y = 0 (static,
    cold, injecting v0) and y = H (moving at U0, hot, sucking v0), periodic x,
    no buoyancy, kinetic rates 1. Re = H v0 / nu unless s_nu is given, in
    which case v0 = Re nu / H and U0 = v0 (the convergence study fixes Re and
    s_nu and keeps the paper's u0 = v0)."""
    if s_nu is None:
        nu = H * v0 / Re
    else:
        nu = (1.0 / s_nu - 0.5) * CS2
        v0 = Re * nu / H
        U0 = v0
    alpha = nu / Pr
    walls = [Wall(0.0, v0, DIRICHLET, T_c, NEE), Wall(U0, v0, DIRICHLET, T_h, NEE)]
    flags = np.zeros((H + 1, nx), np.uint8)
    flags[0, :] = 1
    flags[-1, :] = 2
    return Case("porous_couette_nee", nx, H + 1, True, False, flags, walls, nu=nu, alpha=alpha,
                T0=0.5 * (T_h + T_c), delta_T=T_h - T_c, L=float(H),
                meta=dict(Re=Re, Pr=Pr, U0=U0, v0=v0, T_h=T_h, T_c=T_c, H=H, nodes=True), **KINETIC_ONE)


def porous_couette_nee_exact(case: Case):
    """Eqs. 36-37 on the nodes 0..H."""
    m = case.meta
    y = node_y(m["H"])
    Re, Pr = m["Re"], m["Pr"]
    ux = m["U0"] * np.expm1(Re * y) / np.expm1(Re)
    T = m["T_c"] + (m["T_h"] - m["T_c"]) * np.expm1(Pr * Re * y) / np.expm1(Pr * Re)
    return ux, T


def cavity_nee(n: int = 64, Ra: float = 1e3, Pr: float = 0.71, Ma: float = 0.1, T_h: float = 1.0, T_c: float = 0.0,
               noise: float = 0.0, seed: int = 0, kinetic=None) -> Case:
    """Sec. 3.4 as the paper sets it up: (n + 1) x (n + 1) nodes, walls on the
    boundary nodes (non-equilibrium extrapolation): left hot, right cold, top
    and bottom adiabatic, all static; L = n. Corner nodes belong to the side
    walls."""
    dT = T_h - T_c
    nu, alpha, g_beta = convection_params(float(n), Ra, Pr, Ma, dT)
    walls = [Wall(0, 0, DIRICHLET, T_h, NEE), Wall(0, 0, DIRICHLET, T_c, NEE), Wall(0, 0, ADIABATIC, 0.0, NEE),
             Wall(0, 0, ADIABATIC, 0.0, NEE)]
    flags = np.zeros((n + 1, n + 1), np.uint8)
    flags[0, :] = 3
    flags[-1, :] = 4
    flags[:, 0] = 1
    flags[:, -1] = 2
    T0 = 0.5 * (T_h + T_c)
    Ti = np.full(flags.shape, T0)
    if noise:
        Ti += noise * (2.0 * uniform01(seed, Ti.size).reshape(Ti.shape) - 1.0)
    kin = dict(KINETIC_CONVECTION if kinetic is None else kinetic)
    return Case("cavity_nee", n + 1, n + 1, False, False, flags, walls, nu=nu, alpha=alpha, g_beta=g_beta, T0=T0,
                delta_T=dT, T_init=Ti, L=float(n), meta=dict(Ra=Ra, Pr=Pr, Ma=Ma, nodes=True), **kin)


def lid_cavity_nee(n: int = 192, Re: float = 1000.0, u0: float = 0.1, kinetic=None) -> Case:
    """Sec. 3.2 as the paper sets it up: lid-driven cavity on (n + 1) x (n + 1)
    nodes, walls on the boundary nodes (non-equilibrium extrapolation), the top
    wall moving at (u0, 0), the others static; L = n, nu = L u0 / Re; s_e = 1.6,
    s_q = 1.2, s_eps = 1.8 as the paper lists them. Corner nodes belong to the
    static side walls. Isothermal (no buoyancy, uniform T)."""
    nu = n * u0 / Re
    walls = [Wall(0, 0, ADIABATIC, 0.0, NEE), Wall(0, 0, ADIABATIC, 0.0, NEE), Wall(0, 0, ADIABATIC, 0.0, NEE),
             Wall(u0, 0, ADIABATIC, 0.0, NEE)]
    flags = np.zeros((n + 1, n + 1), np.uint8)
    flags[0, :] = 3
    flags[-1, :] = 4
    flags[:, 0] = 1
    flags[:, -1] = 2
    kin = dict(KINETIC_CONVECTION if kinetic is None else kinetic)
    return Case("lid_cavity_nee", n + 1, n + 1, False, False, flags, walls, nu=nu, alpha=nu / 0.71, T0=0.5,
                L=float(n), meta=dict(Re=Re, u0=u0, nodes=True), **kin)


def with_d2q9_temperature(case: Case, theta: float = 1.0, zeta_q: float = 1.0, zeta_eps: float = 1.0) -> Case:
    """The same problem solved with the D2Q9 temperature model of Eqs. 31-33
    (same alpha; zeta_e and zeta_nu kept). The paper gives no zeta_q, zeta_eps
    for this model; they default to 1, as the paper sets the rates it leaves
    free in Secs. 3.1 and 3.3. (With zeta_nu = zeta_eps = 1.9 the model goes
    unstable on the Rayleigh-Benard workload, the oracle included.)"""
    return replace(case, thermal_q=9, theta=float(theta), zeta_q=float(zeta_q), zeta_eps=float(zeta_eps))


def with_bgk(case: Case) -> Case:
    """The same problem with single-relaxation-time (BGK) collisions: omega
    from nu, zeta from alpha; the other kinetic rates are unused."""
    return replace(case, collision=1)


def with_equal_rates(case: Case) -> Case:
    """MRT with every flow rate set to s_nu and every temperature rate set to
    zeta_alpha (both from the transport coefficients): mathematically the BGK
    collision of the same problem."""
    s_nu = 1.0 / (0.5 + 3.0 * case.nu)
    cs_T2 = 1.0 / 3.0 if case.thermal_q == 9 else 0.5 * case.varpi
    z_a = 1.0 / (0.5 + case.alpha / cs_T2)
    return replace(case, collision=0, s_e=s_nu, s_q=s_nu, s_eps=s_nu, zeta_e=z_a, zeta_nu=z_a, zeta_q=z_a,
                   zeta_eps=z_a)
