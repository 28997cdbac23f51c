"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Nothing here re-types the oracle's formulas. Each check uses an independent
construction: the basis vectors built from the velocity set (Eqs. 5, 12),
exact integer identities, textbook special cases written in velocity space,
the linearised update built from the general MRT definition, closed-form
steady solutions, and values printed in the paper (tests/golden/).
"""
import math
import os

import numpy as np
import pytest

import lbm_cases as lc
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _velocities_eq5():
    """D2Q9 velocities from the trigonometric definition of Eq. 5 (c = 1)."""
    e = [(0.0, 0.0)]
    for i in range(1, 5):
        a = (i - 1) * math.pi / 2
        e.append((math.cos(a), math.sin(a)))
    for i in range(5, 9):
        a = (2 * i - 9) * math.pi / 4
        e.append((math.sqrt(2) * math.cos(a), math.sqrt(2) * math.sin(a)))
    return np.rint(np.array(e)).astype(int)


def _basis_eq12(e):
    ex, ey = e[:, 0].astype(float), e[:, 1].astype(float)
    return np.array([np.ones(9), ex, ey, ex**2 + ey**2, ex**2 - ey**2, ex * ey, ex**2 * ey,
                     ex * ey**2, ex**2 * ey**2])


def _basis_eq26(e):
    ex, ey = e[:5, 0].astype(float), e[:5, 1].astype(float)
    return np.array([np.ones(5), ex, ey, ex**2 + ey**2, ex**2 - ey**2])


E = _velocities_eq5()
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


# ------------------------------------------------------------------ tables --

def test_velocities_match_eq5():
    t = oracle.tables()
    assert np.array_equal(t["ex"], E[:, 0]) and np.array_equal(t["ey"], E[:, 1])


def test_M_rows_are_the_eq12_basis():
    assert np.array_equal(oracle.tables()["M"], _basis_eq12(E))


def test_N_rows_are_the_eq26_basis():
    assert np.array_equal(oracle.tables()["N"], _basis_eq26(E))


def test_inverse_tables_exact_in_integers():
    t = oracle.tables()
    M4 = (4 * t["Minv"]).astype(np.int64)
    N4 = (4 * t["Ninv"]).astype(np.int64)
    assert np.array_equal(4 * t["Minv"], M4) and np.array_equal(4 * t["Ninv"], N4)
    Mi = t["M"].astype(np.int64)
    Ni = t["N"].astype(np.int64)
    assert np.array_equal(Mi @ M4, 4 * np.eye(9, dtype=np.int64))
    assert np.array_equal(M4 @ Mi, 4 * np.eye(9, dtype=np.int64))
    assert np.array_equal(Ni @ N4, 4 * np.eye(5, dtype=np.int64))
    assert np.array_equal(N4 @ Ni, 4 * np.eye(5, dtype=np.int64))


def test_weights_are_isotropic():
    w = oracle.tables()["w"]
    assert np.allclose(w, W, rtol=0, atol=1e-16)
    ex, ey = E[:, 0], E[:, 1]
    assert abs(w.sum() - 1) < 1e-15
    assert abs((w * ex * ex).sum() - 1 / 3) < 1e-15  # c_s^2 = 1/3 (Sec. 2.1)
    assert abs((w * ex * ey).sum()) < 1e-15
    assert abs((w * ex**4).sum() - 3 * (1 / 3) ** 2) < 1e-15
    assert abs((w * ex**2 * ey**2).sum() - (1 / 3) ** 2) < 1e-15


# --------------------------------------------------------------- collision --

def _random_node(rng, amp=0.05):
    f = W * (1 + amp * rng.standard_normal(9))
    g = np.array([0.5, 0.125, 0.125, 0.125, 0.125]) * (0.7 + amp * rng.standard_normal(5))
    return f, g


def test_collision_conserves_mass_momentum_and_T():
    rng = np.random.default_rng(1)
    for _ in range(50):
        s = rng.uniform(0.1, 1.9, 9)
        z = rng.uniform(0.1, 1.9, 5)
        gb, T0 = rng.uniform(-1e-2, 1e-2), rng.uniform(0, 1)
        ax, ay = rng.uniform(-1e-3, 1e-3, 2)
        r = oracle.make_rates(s, z, g_beta=gb, T0=T0, ax=ax, ay=ay)
        f, g = _random_node(rng)
        fs, gs, (rho, ux, uy, T) = oracle.collide_node(r, f, g)
        Fx, Fy = ax, ay + gb * (g.sum() - T0)
        # Eq. 18 and the conserved moments of Sec. 2.1: mass unchanged, momentum
        # changed by exactly rho0 F per step; T = n0 unchanged (Sec. 2.2).
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert abs((E[:, 0] * fs).sum() - (E[:, 0] * f).sum() - Fx) < 1e-15
        assert abs((E[:, 1] * fs).sum() - (E[:, 1] * f).sum() - Fy) < 1e-15
        assert abs(gs.sum() - g.sum()) < 1e-15
        assert abs(T - g.sum()) < 1e-15 and abs(rho - f.sum()) < 1e-15


def _bgk_guo(f, g, omega, omega_T, gb, T0, ax, ay, varpi):
    """Textbook single-relaxation-time update in velocity space: incompressible
    equilibrium (He & Luo 1997) with Guo-Zheng-Shi (2002) forcing for the flow,
    and the D2Q5 equilibrium of Eq. 30 for temperature."""
    T = g.sum()
    F = np.array([ax, ay + gb * (T - T0)])
    rho = f.sum()
    u = E.T @ f + 0.5 * F
    eu = E @ u
    feq = W * (rho + 3 * eu + 4.5 * eu**2 - 1.5 * (u @ u))
    S = W * (3 * (E - u) @ F + 9 * eu * (E @ F))
    fs = f - omega * (f - feq) + (1 - 0.5 * omega) * S
    geq = np.array([(1 - varpi) * T] + [0.25 * varpi * T + 0.5 * (E[i] @ u) * T for i in range(1, 5)])
    gs = g - omega_T * (g - geq)
    return fs, gs


@pytest.mark.parametrize("omega,omega_T", [(1.0, 1.0), (0.6, 1.3), (1.85, 0.9)])
def test_equal_rates_reduce_to_bgk_with_guo_forcing(omega, omega_T):
    rng = np.random.default_rng(2)
    for _ in range(20):
        gb, T0, ax, ay = 3e-3, 0.4, 2e-4, -1e-4
        r = oracle.make_rates([omega] * 9, [omega_T] * 5, g_beta=gb, T0=T0, ax=ax, ay=ay)
        f, g = _random_node(rng, amp=0.2)
        fs, gs, _ = oracle.collide_node(r, f, g)
        fb, gbk = _bgk_guo(f, g, omega, omega_T, gb, T0, ax, ay, 0.5)
        assert np.abs(fs - fb).max() < 1e-15
        assert np.abs(gs - gbk).max() < 1e-15


def test_printed_s8_breaks_the_bgk_limit():
    """Reading A2: with the S~_8 printed in Eq. 17 the equal-rate collision no
    longer equals BGK with Guo forcing, while the form derived from M S does
    (previous test). The difference is O(u F)."""
    rng = np.random.default_rng(3)
    f, g = _random_node(rng, amp=0.2)
    kw = dict(g_beta=5e-2, T0=0.1, ax=3e-2, ay=-2e-2)
    r = oracle.make_rates([0.7] * 9, [1.0] * 5, s8_literal=True, **kw)
    fs, _, _ = oracle.collide_node(r, f, g)
    fb, _ = _bgk_guo(f, g, 0.7, 1.0, kw["g_beta"], kw["T0"], kw["ax"], kw["ay"], 0.5)
    assert np.abs(fs - fb).max() > 1e-6


def test_rates_of_irrelevant_conserved_moments_do_not_matter():
    """s0, s1, s2 (Eq. 20) and zeta0 (Eq. 29) act on conserved moments; with the
    source of Eq. 17 their values drop out of Eq. 8 and Eq. 24."""
    rng = np.random.default_rng(4)
    f, g = _random_node(rng, amp=0.1)
    base = [1.0, 1.0, 1.0, 1.3, 1.6, 1.6, 1.1, 1.1, 0.8]
    out = []
    for s012, z0 in [(1.0, 1.0), (0.3, 1.7), (1.9, 0.2)]:
        s = list(base); s[0] = s[1] = s[2] = s012
        r = oracle.make_rates(s, [z0, 1.2, 1.2, 1.5, 1.7], g_beta=1e-2, T0=0.3, ax=1e-3)
        out.append(oracle.collide_node(r, f, g)[:2])
    for fs, gs in out[1:]:
        assert np.abs(fs - out[0][0]).max() < 1e-15 and np.abs(gs - out[0][1]).max() < 1e-15


# ---------------------------------------------------- linearised dynamics --

def _linear_step(df, dg, s, z, gb, T0, varpi):
    """One step of the MRT update of Eqs. 7-9 and 23-25 linearised about the
    rest state (rho = 1, u = 0, T = T0), built in velocity space from the general
    definition with this test's own matrices (Eqs. 12, 26; inverses by numpy).
    The stored state is post-collision, so a step streams (pull) and then collides."""
    df = np.stack([np.roll(df[i], (E[i, 1], E[i, 0]), (0, 1)) for i in range(9)])
    dg = np.stack([np.roll(dg[i], (E[i, 1], E[i, 0]), (0, 1)) for i in range(5)])
    M = _basis_eq12(E); Mi = np.linalg.inv(M)
    N = _basis_eq26(E); Ni = np.linalg.inv(N)
    Lam = np.diag(s); Q = np.diag(z)
    drho = df.sum(0); dT = dg.sum(0)
    Fy = gb * dT
    ux = np.tensordot(E[:, 0], df, 1)
    uy = np.tensordot(E[:, 1], df, 1) + 0.5 * Fy
    eu = E[:, 0, None, None] * ux + E[:, 1, None, None] * uy
    feq = W[:, None, None] * (drho + 3 * eu)
    S = W[:, None, None] * 3 * (E[:, 1, None, None] * Fy)
    A = Mi @ Lam @ M
    B = Mi @ (np.eye(9) - 0.5 * Lam) @ M
    fs = df - np.tensordot(A, df - feq, 1) + np.tensordot(B, S, 1)
    wT = np.array([1 - varpi] + [varpi / 4] * 4)
    geq = wT[:, None, None] * dT + 0.5 * eu[:5] * T0
    gs = dg - np.tensordot(Ni @ Q @ N, dg - geq, 1)
    return fs, gs


def test_one_step_matches_linearised_mrt_update():
    nx, ny = 7, 6
    rates = dict(s_e=1.37, s_q=0.83, s_eps=1.61, zeta_e=1.23, zeta_nu=0.71)
    nu, alpha, gb, T0, varpi = 0.043, 0.071, 0.02, 0.6, 0.5
    case = lc.periodic_box(nx, ny, nu=nu, alpha=alpha, g_beta=gb, T0=T0, kinetic=rates)
    o = oracle.OracleLattice(case)
    rng = np.random.default_rng(5)
    eps = 1e-6
    df = eps * rng.standard_normal((9, ny, nx))
    dg = eps * rng.standard_normal((5, ny, nx))
    wT = np.array([1 - varpi] + [varpi / 4] * 4)
    o.set_populations(W[:, None, None] + df, wT[:, None, None] * T0 + dg)
    o.step(1)
    f1, g1 = o.populations()
    s_nu = 1 / (0.5 + 3 * nu)
    z_a = 1 / (0.5 + alpha / (varpi / 2))
    s = [1, 1, 1, rates["s_e"], s_nu, s_nu, rates["s_q"], rates["s_q"], rates["s_eps"]]
    z = [1, z_a, z_a, rates["zeta_e"], rates["zeta_nu"]]
    lf, lg = _linear_step(df, dg, s, z, gb, T0, varpi)
    # the neglected terms are O(eps^2); a wrong matrix entry or rate gives O(eps)
    assert np.abs((f1 - W[:, None, None]) - lf).max() < 50 * eps**2
    assert np.abs((g1 - wT[:, None, None] * T0) - lg).max() < 50 * eps**2


def _mode_decay(case, init_f, init_g, read, k_vec, n_settle=150, n_meas=40):
    o = oracle.OracleLattice(case)
    o.set_populations(init_f, init_g)
    o.step(n_settle)
    a0 = read(o)
    o.step(n_meas)
    a1 = read(o)
    return (a1 / a0) ** (1.0 / n_meas)


def test_shear_wave_decays_at_the_eigenvalue_and_the_paper_viscosity():
    """A transverse velocity wave decays per step by the hydrodynamic eigenvalue
    of the linearised update, which tends to exp(-nu k^2) with
    nu = c_s^2 (1/s_nu - 1/2) (Sec. 2.1)."""
    N = 32
    rates = dict(s_e=1.4, s_q=1.15, s_eps=1.7, zeta_e=1.0, zeta_nu=1.0)
    nu = 0.02
    case = lc.periodic_box(2, N, nu=nu, kinetic=rates)
    k = 2 * np.pi / N
    y = np.arange(N)
    ux = 1e-5 * np.sin(k * y)[:, None] * np.ones((1, 2))
    f0 = W[:, None, None] * (1 + 3 * E[:, 0, None, None] * ux)
    g0 = np.zeros((5, N, 2))

    def read(o):
        u = o.macro()[1][:, 0]
        return (u * np.exp(-1j * k * y)).sum()

    lam = _mode_decay(case, f0, g0, read, k).real
    # brute force: eigenvalues of the linearised single-mode update
    s_nu = 1 / (0.5 + 3 * nu)
    s = [1, 1, 1, rates["s_e"], s_nu, s_nu, rates["s_q"], rates["s_q"], rates["s_eps"]]
    M = _basis_eq12(E); Mi = np.linalg.inv(M)
    Eq = W[:, None] * (1 + 3 * (E @ E.T))
    C = np.eye(9) - Mi @ np.diag(s) @ M @ (np.eye(9) - Eq)
    Lk = np.diag(np.exp(-1j * k * E[:, 1])) @ C
    ev = np.linalg.eigvals(Lk)
    lam_h = ev[np.argmin(np.abs(ev - np.exp(-nu * k * k)))]
    assert abs(lam - lam_h) < 1e-10
    nu_meas = -np.log(lam) / k**2
    assert abs(nu_meas - nu) / nu < 5e-3


def test_thermal_wave_decays_at_the_paper_diffusivity():
    """A temperature wave at rest decays by the eigenvalue of the linearised D2Q5
    update, close to exp(-alpha k^2) with alpha = (varpi/2)(1/zeta_alpha - 1/2)
    (Sec. 2.2)."""
    N = 32
    alpha, varpi = 0.03, 0.5
    rates = dict(s_e=1.0, s_q=1.0, s_eps=1.0, zeta_e=1.35, zeta_nu=0.85)
    case = lc.periodic_box(N, 2, alpha=alpha, kinetic=rates)
    k = 2 * np.pi / N
    x = np.arange(N)
    T = 1e-3 * np.sin(k * x)[None, :] * np.ones((2, 1)) + 0.5
    wT = np.array([1 - varpi] + [varpi / 4] * 4)
    f0 = W[:, None, None] * np.ones((9, 2, N))
    g0 = wT[:, None, None] * T[None]

    def read(o):
        t = o.macro()[3][0, :] - 0.5
        return (t * np.exp(-1j * k * x)).sum()

    lam = _mode_decay(case, f0, g0, read, k).real
    z_a = 1 / (0.5 + alpha / (varpi / 2))
    z = [1, z_a, z_a, rates["zeta_e"], rates["zeta_nu"]]
    Nm = _basis_eq26(E); Ni = np.linalg.inv(Nm)
    EqT = wT[:, None] * np.ones((1, 5))
    C = np.eye(5) - Ni @ np.diag(z) @ Nm @ (np.eye(5) - EqT)
    Lk = np.diag(np.exp(-1j * k * E[:5, 0])) @ C
    ev = np.linalg.eigvals(Lk)
    lam_h = ev[np.argmin(np.abs(ev - np.exp(-alpha * k * k)))]
    assert abs(lam - lam_h) < 1e-10
    assert abs(-np.log(lam) / k**2 - alpha) / alpha < 5e-3


# ---------------------------------------------------------- closed forms --

def _run_to_steady(o, chunk, tol, max_chunks):
    o.residual()
    r = np.inf
    for _ in range(max_chunks):
        o.step(chunk)
        r = o.residual()
        if r < tol:
            break
    return r


def test_couette_with_conduction_is_linear():
    """Plane Couette flow between halfway bounce-back walls and conduction between
    anti-bounce-back walls: the steady u_x and T are linear in y."""
    c = lc.couette(H=12, nx=3, U0=0.04, nu=0.09, alpha=0.07)
    o = oracle.OracleLattice(c)
    r = _run_to_steady(o, 2000, 1e-14, 60)
    assert r < 1e-12
    rho, ux, uy, T = o.macro()
    y = lc.fluid_y(12)
    assert np.abs(ux[1:-1] - (0.04 * y)[:, None]).max() < 1e-12
    assert np.abs(T[1:-1] - y[:, None]).max() < 1e-12
    assert np.abs(uy[1:-1]).max() < 1e-14


def test_poiseuille_profile_with_magic_rate_pair():
    """Force-driven channel (Sec. 3.1, Eq. 34). With (1/s_nu - 1/2)(1/s_q - 1/2)
    = 3/16 halfway bounce-back places the wall exactly half-way, so the steady
    nodal profile is the exact parabola."""
    H, ax = 20, 1e-6
    for s_nu in (1.0, 1.754):
        nu = (1 / s_nu - 0.5) / 3
        s_q = 1 / (0.5 + (3 / 16) / (1 / s_nu - 0.5))
        c = lc.poiseuille(H=H, nx=2, ax=ax, nu=nu,
                          kinetic=dict(s_e=1.2, s_q=s_q, s_eps=1.3, zeta_e=1, zeta_nu=1))
        o = oracle.OracleLattice(c)
        o.residual()
        o.step(60000)
        ux = o.macro()[1][1:-1, 0]
        y = np.arange(H) + 0.5
        exact = ax / (2 * nu) * y * (H - y)  # Eq. 34 with l_c = H/2, shifted to 0 <= y <= H
        assert np.abs(ux - exact).max() / exact.max() < 1e-9


def _porous_errors(H):
    c = lc.porous_couette(H=H, nx=2)
    o = oracle.OracleLattice(c)
    _run_to_steady(o, 500, 1e-12, 400)
    rho, ux, uy, T = o.macro()
    ue, Te = lc.porous_couette_exact(c)
    u_num = np.stack([ux[1:-1, 0], uy[1:-1, 0]], 1)
    u_ex = np.stack([ue, np.full(H, c.meta["v0"])], 1)
    Eu = oracle.relative_global_error(u_num, u_ex)  # Eq. 35
    ET = oracle.relative_global_error(T[1:-1, 0], Te)  # Eq. 38
    return Eu, ET, o, c


def test_injection_channel_second_order_convergence():
    """Sec. 3.3, Eqs. 36-38: the oracle converges to the closed-form profiles at
    second order; the paper reports slopes 1.967 (u) and 1.9948 (T)."""
    golden = dict(np.loadtxt(os.path.join(GOLDEN, "sec33_convergence.txt"), dtype=str))
    Hs = [16, 32, 64]
    errs = np.array([_porous_errors(H)[:2] for H in Hs])
    slopes = np.polyfit(np.log(1.0 / np.array(Hs)), np.log(errs), 1)[0]
    for q, sl in zip("uT", slopes):
        assert abs(sl - float(golden[q])) < 0.15, (q, sl)
    assert errs[-1, 0] < 2e-3 and errs[-1, 1] < 1e-3


def test_injection_channel_conserves_mass():
    """The injecting bottom wall adds rho0 v0 per column per step and the top
    wall removes the same amount, so total mass is constant."""
    c = lc.porous_couette(H=32, nx=4)
    o = oracle.OracleLattice(c)
    m0 = o.populations()[0].sum()
    o.step(3000)
    assert abs(o.populations()[0].sum() - m0) / m0 < 1e-13


def test_conduction_cavity_nusselt_is_one():
    """Without buoyancy the steady cavity temperature is linear between the
    isothermal walls, so the Nusselt number of Eq. 39 is exactly 1."""
    c = lc.cavity(n=16, Ra=1e3, noise=0.0).with_(g_beta=0.0)
    o = oracle.OracleLattice(c)
    _run_to_steady(o, 2000, 1e-14, 100)
    assert abs(o.nusselt(0) - 1) < 1e-11 and abs(o.nusselt(1) - 1) < 1e-11
    assert np.isnan(o.nusselt(2))  # adiabatic wall: no fixed wall temperature


def test_conduction_channel_nusselt_on_horizontal_walls():
    """Steady conduction between a hot bottom and a cold top plate: both walls
    carry the conductive flux, Nu = 1 with L = H and dT = T_bot - T_top."""
    c = lc.couette(H=10, nx=2, U0=0.0, T_bot=1.0, T_top=0.25)
    o = oracle.OracleLattice(c)
    _run_to_steady(o, 2000, 1e-14, 100)
    assert abs(o.nusselt(2, L=10.0, dT=0.75) - 1) < 1e-11
    assert abs(o.nusselt(3, L=10.0, dT=0.75) - 1) < 1e-11
    assert abs(o.nusselt(2, L=5.0, dT=0.75) - 0.5) < 1e-11


@pytest.mark.slow
def test_cavity_ra1e3_nusselt_against_table3():
    """Loose physical pin: mean Nu at Ra = 1e3 against the paper's 1.1161
    (Table 3), on a 32^2 grid with halfway walls."""
    row = np.loadtxt(os.path.join(GOLDEN, "table3_cavity.txt"))[0]
    c = lc.cavity(n=32, Ra=1e3)
    o = oracle.OracleLattice(c, threads=min(8, os.cpu_count() or 1))
    _run_to_steady(o, 1000, 1e-9, 100)
    for side in (0, 1):
        assert abs(o.nusselt(side) - row[5]) / row[5] < 5e-3


def test_residual_of_a_rescaled_temperature():
    """Reading A9: scaling T by c everywhere (u unchanged, no buoyancy, no walls)
    gives R = |c - 1| / c; an unchanged state gives 0; the first call gives inf."""
    Ti = 0.5 + 0.1 * lc.uniform01(7, 30).reshape(5, 6)
    c = lc.periodic_box(6, 5, T_init=Ti)
    o = oracle.OracleLattice(c)
    f, g = lc.random_state(c, seed=3)
    o.set_populations(f, g)
    o.step(3)
    assert np.isinf(o.residual())
    f, g = o.populations()
    o.set_populations(f, 1.25 * g)
    R = o.residual()
    assert abs(R - 0.25 / 1.25) < 1e-14
    assert o.residual() == 0.0


def test_residual_of_a_rescaled_velocity():
    """Reading A9 for the velocity: with no force, u = sum e f, so replacing
    f by w + c (f - w) scales u by c everywhere and leaves T alone; then
    R = |c - 1| / c from the velocity part."""
    c = lc.periodic_box(6, 5, T0=0.4)
    o = oracle.OracleLattice(c)
    f, g = lc.random_state(c, seed=4)
    o.set_populations(f, g)
    o.step(3)
    assert np.isinf(o.residual())
    f, g = o.populations()
    w = W[:, None, None]
    o.set_populations(w + 1.5 * (f - w), g)
    assert abs(o.residual() - 0.5 / 1.5) < 1e-13


def test_oracle_rejects_open_edges_and_unknown_walls():
    c = lc.couette(H=4, nx=3)
    with pytest.raises(ValueError):
        oracle.OracleLattice(c.with_(periodic_x=False))
    bad = c.flags.copy(); bad[0, 0] = 9
    with pytest.raises(ValueError):
        oracle.OracleLattice(c.with_(flags=bad))


def _bgk_guo_compressible(f, g, omega, gb, T0, ax, ay):
    """Textbook single-relaxation-time update with the standard (compressible)
    equilibrium w_i rho [1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u^2], u = (sum e f + F rho/2) / rho,
    and the Guo-Zheng-Shi forcing term with rho."""
    T = g.sum()
    F = np.array([ax, ay + gb * (T - T0)])
    rho = f.sum()
    u = (E.T @ f + 0.5 * rho * F) / rho
    eu = E @ u
    feq = W * rho * (1 + 3 * eu + 4.5 * eu**2 - 1.5 * (u @ u))
    S = W * rho * (3 * (E - u) @ F + 9 * eu * (E @ F))
    return f - omega * (f - feq) + (1 - 0.5 * omega) * S


@pytest.mark.parametrize("omega", [0.7, 1.0, 1.6])
def test_rho_in_u_ablation_reduces_to_the_standard_equilibrium(omega):
    """The alternative to reading A1 (rho everywhere, as Eqs. 16-17 and 19 are
    printed): with equal rates it is BGK with the standard compressible
    equilibrium and Guo forcing with rho (not the incompressible one), so
    the two readings differ by O((rho - rho0) u) on states with rho != 1."""
    rng = np.random.default_rng(9)
    kw = dict(g_beta=4e-3, T0=0.3, ax=3e-4, ay=-2e-4)
    for _ in range(20):
        f = W * (1.0 + 0.1 * rng.standard_normal()) * (1 + 0.2 * rng.standard_normal(9))
        g = np.array([0.5, 0.125, 0.125, 0.125, 0.125]) * (0.6 + 0.2 * rng.standard_normal(5))
        alt = oracle.make_rates([omega] * 9, [1.0] * 5, rho_in_u=True, **kw)
        fs, _, (rho, ux, uy, T) = oracle.collide_node(alt, f, g)
        want = _bgk_guo_compressible(f, g, omega, kw["g_beta"], kw["T0"], kw["ax"], kw["ay"])
        assert np.abs(fs - want).max() < 1e-15
        # momentum changes by rho F under this reading
        Fy = kw["ay"] + kw["g_beta"] * (g.sum() - kw["T0"])
        assert abs(E[:, 0] @ fs - E[:, 0] @ f - f.sum() * kw["ax"]) < 1e-15
        assert abs(E[:, 1] @ fs - E[:, 1] @ f - f.sum() * Fy) < 1e-15
        base = oracle.make_rates([omega] * 9, [1.0] * 5, **kw)
        fb, _, _ = oracle.collide_node(base, f, g)
        if abs(f.sum() - 1.0) > 1e-3:
            assert np.abs(fs - fb).max() > 1e-9


def test_rho_in_u_ablation_changes_the_cavity_little():
    """On the Sec. 3.4 cavity (Ra = 1e4, 24^2, 3000 steps) the two readings
    agree to O(Ma^2): density stays within about 1e-3 of rho0, and u and T
    differ by 3.5e-4 (of max |u|) and 1.9e-4 (of delta T)."""
    c = lc.cavity(n=24, Ra=1e4, noise=1e-3)
    a = oracle.OracleLattice(c)
    b = oracle.OracleLattice(c, rho_in_u=True)
    a.step(3000)
    b.step(3000)
    ra, uxa, uya, Ta = a.macro()
    rb, uxb, uyb, Tb = b.macro()
    umax = max(np.abs(uxa).max(), np.abs(uya).max())
    du = max(np.abs(uxa - uxb).max(), np.abs(uya - uyb).max()) / umax
    assert 0 < du < 5e-3 and np.abs(Ta - Tb).max() < 5e-3


def test_relative_global_error_closed_forms():
    """Eqs. 35/38 read as the global L2 norm: a uniform relative deviation eps
    gives eps; a constant offset c on a field with values v gives
    c sqrt(n) / ||v||; a velocity field is measured over both components; a
    permutation of the nodes changes nothing."""
    rng = np.random.default_rng(5)
    v = rng.uniform(0.5, 2.0, (40, 2))
    assert abs(oracle.relative_global_error(v * 1.003, v) - 0.003) < 1e-15
    assert abs(oracle.relative_global_error(v[:, 0] + 1e-3, v[:, 0]) - 1e-3 * np.sqrt(40) / np.linalg.norm(v[:, 0])) < 1e-15
    d = np.zeros_like(v)
    d[7, 1] = 0.02  # one component of one node
    assert abs(oracle.relative_global_error(v + d, v) - 0.02 / np.linalg.norm(v)) < 1e-15
    p = rng.permutation(40)
    assert oracle.relative_global_error((v + d)[p], v[p]) == oracle.relative_global_error(v + d, v)


def _rb_perturbation_growth(Ra, H=20, periods=2):
    """Growth rate, per thermal diffusion time H^2/alpha, of the x-varying
    kinetic energy of a Rayleigh-Benard cell one critical wavelength wide
    (2 pi / 3.117 H, rounded to whole cells) seeded with small temperature
    noise; measured over the last of `periods` diffusion times. Also returns
    the bottom-wall Nusselt number at the end."""
    nx = int(round(2 * np.pi / 3.117 * H))
    c = lc.rayleigh_benard(nx=nx, H=H, Ra=Ra, sigma=1e-3, seed=1)
    o = oracle.OracleLattice(c, threads=min(4, os.cpu_count() or 1))
    tau = int(H * H / c.alpha)
    E = []
    for _ in range(periods):
        o.step(tau)
        _, ux, uy, _ = o.macro()
        ux, uy = ux[1:-1], uy[1:-1]
        # the x-mean is left out: an x-invariant staggered mode of the lattice
        # (alternating u_y from row to row, ~1e-6) is neutral and carries no heat
        E.append(float(((ux - ux.mean(1, keepdims=True)) ** 2 + (uy - uy.mean(1, keepdims=True)) ** 2).sum()))
    return math.log(E[-1] / E[-2]), o.nusselt(2)


def test_rayleigh_benard_onset_near_1708():
    """Linear stability of a fluid layer between rigid isothermal plates
    (Pellew & Southwell 1940; Chandrasekhar 1961): perturbations decay below
    Ra_c = 1707.76 and grow above it, the critical wavenumber being
    3.117 / H. The oracle's Rayleigh-Benard cell (Sec. 3.4's buoyancy, Eq. 4,
    with the rates of Eq. 40) decays at Ra = 1650 and grows at Ra = 1800,
    and the neutral Ra interpolated between them lies within 3 % of 1707.76
    (measured 1729 at H = 20). Below onset the layer returns to conduction,
    Nu = 1. A wrong sign or factor in the buoyancy force, the forcing terms
    or the viscosity / diffusivity relations moves the onset far from 1708."""
    g_lo, nu_lo = _rb_perturbation_growth(1650.0)
    g_hi, _ = _rb_perturbation_growth(1800.0)
    assert g_lo < 0 < g_hi, (g_lo, g_hi)
    Ra_c = 1650.0 + 150.0 * (-g_lo) / (g_hi - g_lo)
    assert abs(Ra_c - 1707.76) / 1707.76 < 0.03, Ra_c
    assert abs(nu_lo - 1.0) < 1e-4, nu_lo


# ----------------------------------------------- 16-bit storage (ablation) --

def test_round_binary16_matches_numpy_float16():
    """The oracle's binary16 rounding (IEEE 754: 10 fraction bits, ties to
    even, subnormals below 2^-14 in steps of 2^-24) equals NumPy's float16
    conversion on values across the whole range, exact ties included."""
    rng = np.random.default_rng(7)
    xs = rng.standard_normal(20000) * 10.0 ** rng.uniform(-9, 4.5, 20000)
    ties = [1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 2.0 ** -24 * 2.5, 2.0 ** -24 * 3.5, 2.0 ** -14 * (1 + 2.0 ** -11),
            -(1 + 2.0 ** -11), 65504.0, 2.0 ** -25, 3 * 2.0 ** -26]
    for x in list(xs) + ties:
        if abs(x) > 65504:
            continue
        assert oracle.round_binary16(x) == float(np.float16(x)), x


def test_sixteen_bit_storage_floor_does_not_move_with_a_scale():
    """What 16-bit storage of the deviations costs, in FP64 arithmetic
    otherwise: on the 32 x 32 cavity at Ra = 1e4 (Sec. 3.4), 4000 steps from
    rest, the max-norm error is about 1e-2 of max |u| and 7e-3 of delta T (the
    11-bit significand of the stored state, rounded every step), far above
    1e-4; multiplying the deviations by 2^8 or 2^12 before rounding (so that
    none falls into the subnormal range) leaves it within 25 %."""
    case = lc.cavity(n=32, Ra=1e4, noise=1e-3)
    ref = oracle.OracleLattice(case, threads=4)
    ref.step(4000)
    _, ux, uy, T = ref.macro()
    umax = max(np.abs(ux).max(), np.abs(uy).max())
    errs = {}
    for scale in (1.0, 256.0, 4096.0):
        q = oracle.OracleLattice(case, threads=4)
        q.set_storage_rounding(16, scale)
        q.step(4000)
        _, qx, qy, qT = q.macro()
        errs[scale] = (max(np.abs(qx - ux).max(), np.abs(qy - uy).max()) / umax, np.abs(qT - T).max())
    eu, eT = errs[1.0]
    assert 3e-3 < eu < 3e-2 and 2e-3 < eT < 2e-2, errs
    for scale in (256.0, 4096.0):
        assert abs(errs[scale][0] / eu - 1) < 0.25 and abs(errs[scale][1] / eT - 1) < 0.25, errs
    # the ablation is off by default: a lattice without it matches the reference
    q = oracle.OracleLattice(case, threads=4)
    q.step(10)
    r2 = oracle.OracleLattice(case, threads=4)
    r2.set_storage_rounding(0)
    r2.step(10)
    assert all(np.array_equal(a, b) for a, b in zip(q.populations(), r2.populations()))
