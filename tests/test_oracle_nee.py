"""Pins of the oracle's node-based walls with non-equilibrium extrapolation
(Guo, Zheng & Shi 2002), the boundary treatment the paper uses (Sec. 3).

The paper cites the scheme without its formulas; this code reconstructs the
boundary node's pre-collision populations as the equilibrium at the wall
state plus the nearest fluid node's non-equilibrium part, then collides the
node like a fluid node. The paper's error tables therefore pin magnitudes and
trends, not digits: E_u (Eq. 35 as the global L2 norm) within 6 % of Table 2
at every rate and within 15 % in the per-node reading, the ordering in s_nu,
the two-point slope of Table 2 within 0.01, the velocity slope of Sec. 3.3
within 0.02, the near independence of E_u from a_x of Table 1, and the cavity
Nusselt number of Table 3."""
import os

import numpy as np
import pytest

import lbm_cases as lc
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _steady(o, chunk=2000, tol=1e-12, max_chunks=3000):
    o.residual()
    r = np.inf
    for _ in range(max_chunks):
        o.step(chunk)
        r = o.residual()
        if r < tol:
            break
    return r


def _poiseuille_error(H, s_nu, Re=49.4146, ax=None, nee_uf="eq19"):
    """(E_u as the global L2 norm, E_u as summed per-node norms) of the
    channel at steady state; ax follows from Re unless given."""
    nu = (1 / s_nu - 0.5) / 3
    if ax is None:
        ax = 2 * Re * nu**2 / (H / 2) ** 3  # Re = u0 l_c / nu with u0 = ax l_c^2 / (2 nu), l_c = H / 2
    c = lc.poiseuille_nee(H=H, nx=2, ax=ax, s_nu=s_nu)
    o = oracle.OracleLattice(c, nee_uf=nee_uf)
    _steady(o)
    ux = o.macro()[1][:, 0]
    y = np.arange(H + 1)
    ua = ax / (2 * nu) * y * (H - y)  # Eq. 34 on the nodes, walls at y = 0 and y = H
    # Eq. 35 (u_y is zero in both, so the per-node norm is |u_x - u_A|)
    return oracle.relative_global_error(ux, ua), np.abs(ux - ua).sum() / np.abs(ua).sum()


def test_node_wall_rebuild_from_an_equilibrium_state():
    """The scheme's definition on a state it must reproduce exactly: every node
    at the same force-free equilibrium (rho = 1, u0, T0). After streaming, a
    boundary node's fluid neighbour holds that equilibrium, so its
    non-equilibrium part is zero and the rebuilt node is the equilibrium at the
    wall state (1, u_w, T_w) of Eq. 22 and Eq. 30; collision keeps an
    equilibrium, so that is what the node stores after one step, while every
    fluid node keeps (1, u0, T0)."""
    c = lc.porous_couette_nee(H=8, nx=3, Re=10.0, U0=0.02, v0=0.01)
    E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
    W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)

    def feq(u):
        eu = E @ u
        return W * (1 + 3 * eu + 4.5 * eu**2 - 1.5 * (u @ u))

    def geq(T, u):
        return np.array([(1 - c.varpi) * T] + [c.varpi / 4 * T + 0.5 * (E[i] @ u) * T for i in range(1, 5)])

    u0, T0 = np.array([0.013, -0.007]), 0.37
    f = np.broadcast_to(feq(u0)[:, None, None], (9, c.ny, c.nx)).copy()
    g = np.broadcast_to(geq(T0, u0)[:, None, None], (5, c.ny, c.nx)).copy()
    o = oracle.OracleLattice(c)
    o.set_populations(f, g)
    o.step(1)
    f1, g1 = o.populations()
    for row, wall in ((0, c.walls[0]), (c.ny - 1, c.walls[1])):
        uw = np.array([wall.ux, wall.uy])
        assert np.abs(f1[:, row, :] - feq(uw)[:, None]).max() < 1e-15
        assert np.abs(g1[:, row, :] - geq(wall.T, uw)[:, None]).max() < 1e-15
    assert np.abs(f1[:, 1:-1, :] - feq(u0)[:, None, None]).max() < 1e-15
    assert np.abs(g1[:, 1:-1, :] - geq(T0, u0)[:, None, None]).max() < 1e-15


def test_poiseuille_errors_match_table2_in_magnitude_and_order():
    """Measured at dx = 1/30: global-L2 E_u 1.055 / 1.032 / 1.013 x Table 2 for
    s_nu = 1.60 / 1.754 / 1.90, per-node form 1.137 / 1.113 / 1.092 x."""
    tab = np.loadtxt(os.path.join(GOLDEN, "table1_2_poiseuille.txt"))
    errs = []
    for row in tab:
        e30, e30_node = _poiseuille_error(30, row[0])
        assert abs(e30 - row[1]) / row[1] < 0.06, (row[0], e30, row[1])
        assert abs(e30_node - row[1]) / row[1] < 0.15, (row[0], e30_node, row[1])
        errs.append(e30)
    assert errs[0] < errs[1] < errs[2]  # E_u grows with s_nu at fixed Re, as in Table 2
    e60, _ = _poiseuille_error(60, 1.754)
    assert abs(e60 - tab[1, 2]) / tab[1, 2] < 0.06
    # two-point slope between dx = 1/30 and 1/60: Table 2's own is 1.9859, ours 1.9891
    slope = np.log(errs[1] / e60) / np.log(2.0)
    assert abs(slope - np.log(tab[1, 1] / tab[1, 2]) / np.log(2.0)) < 0.01


def test_poiseuille_error_nearly_independent_of_body_force_table1():
    """Table 1: at s_nu = 1.754 and dx = 1/60, E_u moves by 0.6 % as a_x goes
    from 2e-6 to 8e-6 (Re from 49 to 198): the error is a property of the
    walls and the resolution, not of the flow speed. Ours moves by 0.5 %, in
    the other direction. The move comes from the fluid node's velocity inside
    the extrapolated non-equilibrium part: with u_f = (j - F/2)/rho0 instead of
    Eq. 19's (j + F/2)/rho0 the oracle's E_u follows Table 1 to 0.1 % in ratio
    (it falls by 0.54 % where the paper's falls by 0.60 %), which is why
    reading A11 names that detail as the likely difference."""
    e2, _ = _poiseuille_error(60, 1.754, ax=2e-6)
    e8, _ = _poiseuille_error(60, 1.754, ax=8e-6)
    assert abs(e8 / e2 - 1) < 0.01 and abs(e2 - 1.2600e-3) / 1.2600e-3 < 0.06
    assert e8 > e2  # the reading's trend
    m2, _ = _poiseuille_error(60, 1.754, ax=2e-6, nee_uf="minus")
    m8, _ = _poiseuille_error(60, 1.754, ax=8e-6, nee_uf="minus")
    assert m8 < m2  # Table 1's trend
    assert abs((m8 / 1.2524e-3) / (m2 / 1.2600e-3) - 1) < 1e-3


def test_injection_channel_slopes_match_sec33():
    golden = dict(np.loadtxt(os.path.join(GOLDEN, "sec33_convergence.txt"), dtype=str))
    Hs = [30, 60, 90]
    eu, eT = [], []
    for H in Hs:
        c = lc.porous_couette_nee(H=H, nx=2, Re=10, s_nu=0.8)
        o = oracle.OracleLattice(c)
        _steady(o, chunk=1000)
        rho, ux, uy, T = o.macro()
        ue, Te = lc.porous_couette_nee_exact(c)
        u_num = np.stack([ux[:, 0], uy[:, 0]], 1)
        u_ex = np.stack([ue, np.full(H + 1, c.meta["v0"])], 1)
        eu.append(oracle.relative_global_error(u_num, u_ex))  # Eq. 35
        eT.append(oracle.relative_global_error(T[:, 0], Te))  # Eq. 38
        assert np.abs(uy[:, 0] - c.meta["v0"]).max() < 1e-12  # the normal velocity is exact
    su = np.polyfit(np.log(1.0 / np.array(Hs)), np.log(eu), 1)[0]
    sT = np.polyfit(np.log(1.0 / np.array(Hs)), np.log(eT), 1)[0]
    # over dx = 1/30..1/90: 1.957 (1.939 with the per-node form of Eq. 35); over
    # the paper's 1/30..1/150: 1.965 (per-node 1.951) against the printed 1.967
    assert abs(su - float(golden["u"])) < 0.02 and abs(sT - float(golden["T"])) < 0.05, (su, sT)


def test_conduction_cavity_nusselt_is_one_with_node_walls():
    c = lc.cavity_nee(n=16, Ra=1e3).with_(g_beta=0.0)
    o = oracle.OracleLattice(c)
    _steady(o, chunk=2000, tol=1e-14, max_chunks=200)
    assert abs(o.nusselt(0, L=16) - 1) < 1e-10 and abs(o.nusselt(1, L=16) - 1) < 1e-10
    T = o.macro()[3]
    assert np.abs(T[:, 0] - 1).max() < 1e-12 and np.abs(T[:, -1]).max() < 1e-12  # wall nodes hold T_w


@pytest.mark.slow
def test_cavity_ra1e3_node_walls_against_table3():
    row = np.loadtxt(os.path.join(GOLDEN, "table3_cavity.txt"))[0]
    c = lc.cavity_nee(n=64, Ra=1e3)
    o = oracle.OracleLattice(c, threads=min(8, os.cpu_count() or 1))
    _steady(o, chunk=1000, tol=1e-9, max_chunks=200)
    for side in (0, 1):
        assert abs(o.nusselt(side, L=64) - row[5]) / row[5] < 5e-3
