"""Pins of the oracle's D2Q9 temperature model (Eqs. 31-33): the equal-rate
limit is single-relaxation-time in velocity space with the equilibrium of
Eq. 31 (either theta), the temperature is conserved, the linearised update
matches the general MRT definition built here, a temperature wave decays at
alpha = c_s^2 (1/zeta_alpha - 1/2), conduction is linear, and the cavity
Nusselt number matches Table 3."""
import os

import numpy as np
import pytest

import lbm_cases as lc
import oracle
from test_oracle_pins import E, W, _basis_eq12, _random_node

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _geq31(T, u, theta):
    eu = E @ u
    return W * T * (1 + 3 * eu + theta * (4.5 * eu**2 - 1.5 * (u @ u)))


@pytest.mark.parametrize("theta", [0.0, 1.0])
@pytest.mark.parametrize("omega_T", [0.7, 1.0, 1.6])
def test_equal_rates_reduce_to_srt_with_eq31(theta, omega_T):
    rng = np.random.default_rng(8)
    for _ in range(20):
        f = W * (1 + 0.1 * rng.standard_normal(9))
        g = W * (0.6 + 0.1 * rng.standard_normal(9))
        r = oracle.make_rates([1.3] * 9, [omega_T] * 9, g_beta=2e-3, T0=0.4, ax=1e-4, theta=theta)
        fs, gs, (rho, ux, uy, T) = oracle.collide_node(r, f, g)
        u = np.array([ux, uy])
        want = g - omega_T * (g - _geq31(g.sum(), u, theta))
        assert np.abs(gs - want).max() < 1e-15
        assert abs(gs.sum() - g.sum()) < 1e-15


def test_rates_act_on_their_moments_linearised():
    """One step from a small perturbation of rest at T0 on a periodic lattice
    equals the linearised update built from the general definition: streaming,
    then g* = g - M^-1 Q M (g - g_eq_lin), g_eq_lin = w_i (dT + 3 T0 e_i . u)."""
    nx, ny = 6, 7
    case = lc.with_d2q9_temperature(lc.periodic_box(nx, ny, nu=0.05, alpha=0.04, T0=0.6,
                                                    kinetic=dict(s_e=1.2, s_q=1.1, s_eps=1.3, zeta_e=1.25,
                                                                 zeta_nu=0.85)),
                                    theta=1.0, zeta_q=1.45, zeta_eps=0.75)
    o = oracle.OracleLattice(case)
    rng = np.random.default_rng(9)
    eps = 1e-6
    df = eps * rng.standard_normal((9, ny, nx))
    dg = eps * rng.standard_normal((9, ny, nx))
    o.set_populations(W[:, None, None] + df, W[:, None, None] * 0.6 + dg)
    o.step(1)
    _, g1 = o.populations()
    df = np.stack([np.roll(df[i], (E[i, 1], E[i, 0]), (0, 1)) for i in range(9)])
    dg = np.stack([np.roll(dg[i], (E[i, 1], E[i, 0]), (0, 1)) for i in range(9)])
    ux = np.tensordot(E[:, 0], df, 1)
    uy = np.tensordot(E[:, 1], df, 1)
    dT = dg.sum(0)
    eu = E[:, 0, None, None] * ux + E[:, 1, None, None] * uy
    geq = W[:, None, None] * (dT + 3 * 0.6 * eu)
    za = 1 / (0.5 + 0.04 * 3)
    Q = np.diag([1, za, za, 1.25, 0.85, 0.85, 1.45, 1.45, 0.75])
    M = _basis_eq12(E)
    lg = dg - np.tensordot(np.linalg.inv(M) @ Q @ M, dg - geq, 1)
    assert np.abs((g1 - W[:, None, None] * 0.6) - lg).max() < 50 * eps**2


def test_thermal_wave_decays_at_the_d2q9_diffusivity():
    N, alpha = 32, 0.03
    case = lc.with_d2q9_temperature(lc.periodic_box(N, 2, alpha=alpha), zeta_q=1.3, zeta_eps=0.9)
    k = 2 * np.pi / N
    x = np.arange(N)
    T = 0.5 + 1e-3 * np.sin(k * x)[None, :] * np.ones((2, 1))
    o = oracle.OracleLattice(case)
    o.set_populations(W[:, None, None] * np.ones((9, 2, N)), W[:, None, None] * T[None])

    def amp():
        t = o.macro()[3][0, :] - 0.5
        return (t * np.exp(-1j * k * x)).sum()
    o.step(200)
    a0 = amp()
    o.step(40)
    lam = (amp() / a0).real ** (1 / 40)
    za = 1 / (0.5 + alpha * 3)  # alpha = c_s^2 (1/zeta_alpha - 1/2), c_s^2 = 1/3
    Q = np.diag([1, za, za, 1.0, 1.0, 1.0, 1.3, 1.3, 0.9])
    M = _basis_eq12(E)
    C = np.eye(9) - np.linalg.inv(M) @ Q @ M @ (np.eye(9) - W[:, None] * np.ones((1, 9)))
    ev = np.linalg.eigvals(np.diag(np.exp(-1j * k * E[:, 0])) @ C)
    lam_h = ev[np.argmin(np.abs(ev - np.exp(-alpha * k * k)))]
    assert abs(lam - lam_h) < 1e-10
    assert abs(-np.log(lam) / k**2 - alpha) / alpha < 5e-3


def test_conduction_is_linear_with_d2q9_temperature():
    c = lc.with_d2q9_temperature(lc.couette(H=10, nx=3, U0=0.03, alpha=0.06), theta=1.0)
    o = oracle.OracleLattice(c)
    o.residual()
    for _ in range(100):
        o.step(2000)
        if o.residual() < 1e-14:
            break
    T = o.macro()[3][1:-1, 0]
    assert np.abs(T - lc.fluid_y(10)).max() < 1e-12


@pytest.mark.slow
def test_cavity_ra1e3_d2q9_temperature_against_table3():
    row = np.loadtxt(os.path.join(GOLDEN, "table3_cavity.txt"))[0]
    c = lc.with_d2q9_temperature(lc.cavity(n=32, Ra=1e3))
    o = oracle.OracleLattice(c, threads=min(8, os.cpu_count() or 1))
    o.residual()
    for _ in range(100):
        o.step(1000)
        if o.residual() < 1e-9:
            break
    for side in (0, 1):
        assert abs(o.nusselt(side) - row[5]) / row[5] < 5e-3
