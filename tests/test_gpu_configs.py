"""The paper-shaped configurations on the GPU.

* Rayleigh-Benard crop, 256 x 128 fluid cells at the Ra = 1e6, Pr = 0.71
  parameters of the 4096 x 2048 benchmark cell (same nu, alpha, g beta):
  FP64 storage must match the FP64 oracle to 1e-12 (relative max-norm);
  FP32- and FP16-shifted storage state their max-norm errors in u and T.
  That crop's own Rayleigh number is about 244, so it stays conductive.
* Convective Rayleigh-Benard cell, 256 x 128 fluid cells with L = H = 128,
  so its own Ra = 1e6 (Eq. 40 rates, Sec. 3.4), 25,000 steps through onset
  into developed convection (Nu about 7-8): FP64 against the oracle to
  1e-12, FP32/FP16 errors stated and compared with how far the flow itself
  carries a perturbation of FP32 rounding size.
* Differentially heated cavity, 256 x 256, Ra = 1e5, Pr = 0.71, Ma = 0.1,
  2e5 steps in FP64 and FP32 storage: mean Nusselt number on the hot wall
  against the paper's Table 3 (cold wall 4.5273; equal at steady state).
* Porous-plate thermal Couette, 8 x 64 fluid cells, Re = 5, Pr = 0.71,
  Ra = 100, run to residual < 1e-10 in FP64: the profiles against the closed
  forms of Eqs. 36-37 (Sec. 3.3) and against the oracle after the same steps;
  FP32 after the same steps against the oracle.
"""
import os

import numpy as np
import pytest

import lbm_cases as lc
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Max-norm errors after 1000 steps, u in units of the problem's velocity scale
# u_c = Ma c_s and T in units of delta T. This crop keeps the big cell's nu,
# alpha and g beta, so its own Rayleigh number is 1e6 (128/2048)^3 ~ 244: it
# stays conductive and |u| decays (max |u| ~ 1e-6), which is why u is not
# measured against its own maximum. Measured: FP32 u 3e-10, T 2e-7; FP16
# u 2e-5, T 5e-4; bounded with margin.
RB_TOL = {"f32": {"u": 1e-8, "T": 1e-6}, "f16": {"u": 2e-4, "T": 2e-3}}


@pytest.fixture(scope="module")
def rb_crop_oracle():
    case = lc.rayleigh_benard(nx=256, H=128, Ra=1e6, Pr=0.71, Ma=0.1, seed=0, sigma=1e-3, L=2048)
    o = oracle.OracleLattice(case, threads=min(8, os.cpu_count() or 1))
    o.step(1000)
    return case, o.macro(), o.populations()


def test_rb_crop_fp64_matches_oracle(rb_crop_oracle):
    import paper_1510_08224_gb300 as P
    case, mac, pops = rb_crop_oracle
    g = P.Lattice(case, storage="f64")
    g.step(1000)
    f, t = g.populations()
    assert np.abs(f - pops[0]).max() / np.abs(pops[0]).max() <= 1e-12
    assert np.abs(t - pops[1]).max() / np.abs(pops[1]).max() <= 1e-12
    for a, b in zip(g.macro(), mac):
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_rb_crop_reduced_precision_error(rb_crop_oracle, storage):
    import paper_1510_08224_gb300 as P
    case, (_, uxo, uyo, To), _ = rb_crop_oracle
    g = P.Lattice(case, storage=storage)
    g.step(1000)
    _, ux, uy, T = g.macro()
    u_c = case.meta["Ma"] * np.sqrt(1.0 / 3.0)
    eu = max(np.abs(ux - uxo).max(), np.abs(uy - uyo).max()) / u_c
    eT = np.abs(T - To).max() / case.delta_T
    print(f"RB 256x128 crop, {storage}, 1000 steps: max-norm error u {eu:.2e} (of u_c {u_c:.3f}), T {eT:.2e}")
    assert eu <= RB_TOL[storage]["u"] and eT <= RB_TOL[storage]["T"]


# The convective cell: seeded 5e-2 perturbation so that convection sets in
# within the run (onset near 15,000 steps, developed by 20,000). Checked at
# 10,000 steps (the flow still growing) and at 25,000 (developed convection).
RB_CONV_STEPS = (10_000, 25_000)


@pytest.fixture(scope="module")
def rb_convective_oracle():
    """The oracle on the convective cell at both check points, and the same
    oracle started from an initial temperature changed by a relative 6e-8
    (FP32 rounding size): the difference of the two is how far this flow
    carries a rounding-sized perturbation on its own."""
    case = lc.rayleigh_benard(nx=256, H=128, Ra=1e6, Pr=0.71, Ma=0.1, seed=0, sigma=5e-2)
    threads = min(16, os.cpu_count() or 1)
    o = oracle.OracleLattice(case, threads=threads)
    jitter = 1 + 6e-8 * (2 * lc.uniform01(99, case.T_init.size).reshape(case.T_init.shape) - 1)
    o2 = oracle.OracleLattice(case.with_(T_init=case.T_init * jitter), threads=threads)
    snaps, done = [], 0
    for k in RB_CONV_STEPS:
        o.step(k - done)
        o2.step(k - done)
        done = k
        snaps.append(dict(macro=o.macro(), pops=o.populations(), jitter=o2.macro(), nu=o.nusselt(2)))
    return case, snaps


def _conv_errors(case, mac, ref):
    _, ux, uy, T = mac
    _, uxo, uyo, To = ref
    umax = max(np.abs(uxo).max(), np.abs(uyo).max())
    eu = max(np.abs(ux - uxo).max(), np.abs(uy - uyo).max()) / umax
    eT = np.abs(T - To).max() / case.delta_T
    return eu, eT, umax


# FP64 against the oracle: 1e-12 at 10,000 steps; at 25,000 the developed
# convection has amplified every difference (a relative 6e-8 change of the
# initial temperature grows about 40-60 fold by then, oracle against oracle),
# the rounding differences between the two programs' orders of operations
# (about 1e-16 per step) included: 1e-10.
RB_CONV_FP64_TOL = (1e-12, 1e-10)


def test_rb_convective_fp64_matches_oracle(rb_convective_oracle):
    import paper_1510_08224_gb300 as P
    case, snaps = rb_convective_oracle
    u_c = case.meta["Ma"] * np.sqrt(1.0 / 3.0)
    _, uxo, uyo, _ = snaps[1]["macro"]
    # the run reaches developed convection
    assert max(np.abs(uxo).max(), np.abs(uyo).max()) > 0.3 * u_c and snaps[1]["nu"] > 4.0
    g = P.Lattice(case, storage="f64")
    done = 0
    for k, snap, tol in zip(RB_CONV_STEPS, snaps, RB_CONV_FP64_TOL):
        g.step(k - done)
        done = k
        f, t = g.populations()
        pops = snap["pops"]
        ef = np.abs(f - pops[0]).max() / np.abs(pops[0]).max()
        et = np.abs(t - pops[1]).max() / np.abs(pops[1]).max()
        em = max(np.abs(a - b).max() / max(1.0, np.abs(b).max()) for a, b in zip(g.macro(), snap["macro"]))
        print(f"RB 256x128 convective, FP64, {k} steps: populations f {ef:.2e}, g {et:.2e}, fields {em:.2e}")
        assert ef <= tol and et <= tol and em <= tol, (k, ef, et, em)
    assert abs(g.nusselt("bottom") - snaps[1]["nu"]) <= 1e-9 * snaps[1]["nu"]


# Max-norm errors (u of max |u|, T of delta T) at 10,000 and 25,000 steps.
# FP32: the storage rounds every population by about 6e-8 of its deviation at
# every step, and the flow amplifies such changes (the oracle carries a single
# 6e-8 change of the initial temperature to 4e-7 / 2e-8 by 10,000 steps and
# 4e-6 / 3e-6 by 25,000): measured 8.7e-6 / 6.0e-7 and 1.6e-4 / 8.5e-5, with
# the mean Nusselt number on the hot plate within 1e-5 of the oracle's. FP16
# rounds about 8,000 times more per step: at 10,000 steps, with the rolls
# still growing (max |u| = 0.04 u_c), its velocity field has already left the
# oracle's (measured 0.60 of max |u|; T 3.3e-2), and in developed convection
# its plumes sit elsewhere (errors of order one), so at 25,000 steps only the
# character of the flow is checked: finite, convecting, with a Nusselt number
# of developed convection.
RB_CONV_TOL = {"f32": ({"u": 3e-5, "T": 3e-6}, {"u": 5e-4, "T": 3e-4}),
               "f16": ({"u": 1.0, "T": 0.1}, None)}


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_rb_convective_reduced_precision_error(rb_convective_oracle, storage):
    import paper_1510_08224_gb300 as P
    case, snaps = rb_convective_oracle
    g = P.Lattice(case, storage=storage)
    done = 0
    for k, snap, tol in zip(RB_CONV_STEPS, snaps, RB_CONV_TOL[storage]):
        g.step(k - done)
        done = k
        mac = g.macro()
        eu, eT, umax = _conv_errors(case, mac, snap["macro"])
        fu, fT, _ = _conv_errors(case, snap["jitter"], snap["macro"])
        nu = g.nusselt("bottom")
        print(f"RB 256x128 convective (L = 128, Ra 1e6), {storage}, {k} steps: max-norm error u {eu:.2e} "
              f"(of max|u| {umax:.3e}), T {eT:.2e}; Nu bottom {nu:.4f} (oracle {snap['nu']:.4f}); the oracle "
              f"carries a 6e-8 initial change to u {fu:.2e}, T {fT:.2e}")
        if tol is not None:
            assert eu <= tol["u"] and eT <= tol["T"], (k, eu, eT)
        else:
            u_c = case.meta["Ma"] * np.sqrt(1.0 / 3.0)
            assert np.isfinite(mac[1]).all() and max(np.abs(mac[1]).max(), np.abs(mac[2]).max()) > 0.3 * u_c
            assert 4.0 < nu < 15.0


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_cavity_ra1e5_256_nusselt_against_table3(storage):
    import paper_1510_08224_gb300 as P
    row = np.loadtxt(os.path.join(GOLDEN, "table3_cavity.txt"))[2]  # Ra = 1e5
    case = lc.cavity(n=256, Ra=1e5, Pr=0.71, Ma=0.1, seed=0, noise=1e-6)
    g = P.Lattice(case, storage=storage)
    g.step(200_000)
    nu_hot, nu_cold = g.nusselt("left"), g.nusselt("right")
    print(f"cavity 256^2 Ra 1e5 {storage}: Nu hot {nu_hot:.4f} cold {nu_cold:.4f} (Table 3: {row[5]})")
    assert abs(nu_hot - row[5]) / row[5] < 0.01
    assert abs(nu_cold - row[5]) / row[5] < 0.01


def _eu_et(case, ux, uy, T):
    """Eqs. 35 and 38 (relative errors of u and T) against Eqs. 36-37."""
    ue, Te = lc.porous_couette_exact(case)
    u_num = np.stack([ux[1:-1, :].mean(1), uy[1:-1, :].mean(1)], 1)
    u_ex = np.stack([ue, np.full(ue.size, case.meta["v0"])], 1)
    Eu = oracle.relative_global_error(u_num, u_ex)
    ET = oracle.relative_global_error(T[1:-1, :].mean(1), Te)
    return Eu, ET


@pytest.fixture(scope="module")
def injection_channel_steady():
    """FP64 GPU run of the 8 x 64 injection channel to residual < 1e-10
    (checked every 1000 steps); the oracle advanced by the same steps."""
    import paper_1510_08224_gb300 as P
    case = lc.porous_couette(H=64, nx=8)
    g = P.Lattice(case, storage="f64")
    g.residual()
    steps = 0
    r = float("inf")
    while r >= 1e-10 and steps < 400_000:
        g.step(1000)
        steps += 1000
        r = g.residual()
    o = oracle.OracleLattice(case)
    o.step(steps)
    return case, steps, r, g.macro(), o.macro()


def test_injection_channel_fp64_steady_state(injection_channel_steady):
    case, steps, r, gm, om = injection_channel_steady
    assert r < 1e-10
    for a, b in zip(gm, om):
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())
    Eu, ET = _eu_et(case, *gm[1:])
    print(f"injection channel 8x64, FP64, {steps} steps, R {r:.1e}: E_u {Eu:.3e}, E_T {ET:.3e}")
    # second-order error of the halfway walls at H = 64 (the oracle pin's bounds)
    assert Eu < 2e-3 and ET < 1e-3
    # the flow is uniform along the periodic x direction
    assert np.abs(gm[1][1:-1] - gm[1][1:-1, :1]).max() < 1e-12


def test_injection_channel_fp32_against_oracle(injection_channel_steady):
    import paper_1510_08224_gb300 as P
    case, steps, r, gm, om = injection_channel_steady
    g = P.Lattice(case, storage="f32")
    g.step(steps)
    _, ux, uy, T = g.macro()
    _, uxo, uyo, To = om
    umax = max(np.abs(uxo).max(), np.abs(uyo).max())
    eu = max(np.abs(ux - uxo).max(), np.abs(uy - uyo).max()) / umax
    eT = np.abs(T - To).max() / case.delta_T
    print(f"injection channel 8x64, FP32, {steps} steps: max-norm error u {eu:.2e} (of max|u|), T {eT:.2e}")
    assert eu <= 1e-4 and eT <= 1e-4


@pytest.mark.parametrize("row", [0, 1])
def test_table3_with_the_papers_node_walls(row):
    """Table 3 (Sec. 3.4) as the paper computes it: node-based walls with
    non-equilibrium extrapolation, the paper's grid (128^2 at Ra = 1e3, 192^2 at
    Ra = 1e4), FP64, run to a residual below 1e-10. u_x max and u_y max on the
    midlines (in units of alpha / L), the maximum and the mean of the cold-wall
    Nusselt number within 0.5 % of the printed values, and their positions
    within one node."""
    import bench
    import paper_1510_08224_gb300 as P
    vals = np.loadtxt(os.path.join(GOLDEN, "table3_cavity.txt"))[row]
    pos = np.loadtxt(os.path.join(GOLDEN, "table3_positions.txt"))[row]
    Ra, grid = vals[0], int(vals[1])
    case = lc.cavity_nee(n=grid, Ra=Ra)
    g = P.Lattice(case, storage="f64")
    g.residual()
    steps, r = 0, float("inf")
    while r >= 1e-10 and steps < 1_000_000:
        g.step(2000)
        steps += 2000
        r = g.residual()
    assert r < 1e-10
    q = bench.cavity_table3_quantities(case, *g.macro())
    print(f"Ra {Ra:g}, {grid}^2, {steps} steps: {q}")
    for k, v in zip(("ux_max", "uy_max", "Nu_max", "Nu_mean"), vals[2:]):
        assert abs(q[k] - v) / v < 5e-3, (k, q[k], v)
    for k, v in zip(("y_max", "x_max", "y_Nu"), pos[2:]):
        assert abs(q[k] - v) <= 1.0 / grid + 1e-4, (k, q[k], v)
    # the volume form of the Nusselt number agrees with the wall form at steady state
    assert abs(q["Nu_vol"] - q["Nu_mean"]) / q["Nu_mean"] < 1e-2


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
@pytest.mark.parametrize("with_T", [True, False])
def test_initial_state_of_a_lattice_taller_than_one_upload_chunk(storage, with_T):
    """lbm_create uploads T_init in chunks of the staging area (252 rows of an
    8192-wide lattice): a 8192 x 600 periodic box starts at rest from T_init (a
    seeded field) or from T0 everywhere, across the chunk seams. The initial
    populations are the equilibria at (rho0, 0, T) (reading A4) and the
    read-out is taken after the pull (reading A6), so it shows
    (1 - varpi) T(x) + varpi/4 times the sum of T over the four axis
    neighbours, to rounding of the storage."""
    import paper_1510_08224_gb300 as P
    nx, ny = 8192, 600
    T = 0.5 + 0.25 * (2 * lc.uniform01(17, nx * ny).reshape(ny, nx) - 1) if with_T else None
    case = lc.periodic_box(nx, ny, T0=0.5, T_init=T)
    lat = P.Lattice(case, storage=storage)
    rho, ux, uy, Tg = lat.macro()
    if with_T:
        nb = np.roll(T, 1, 0) + np.roll(T, -1, 0) + np.roll(T, 1, 1) + np.roll(T, -1, 1)
        Te = (1 - case.varpi) * T + case.varpi / 4 * nb
    else:
        Te = np.full((ny, nx), 0.5)
    tol = {"f64": 1e-15, "f32": 1e-7, "f16": 1e-3}[storage]
    assert np.abs(Tg - Te).max() <= tol
    assert np.abs(rho - 1).max() <= tol and np.abs(ux).max() <= 1e-15 and np.abs(uy).max() <= 1e-15
    lat.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_large_channel_rows_against_oracle(storage):
    """A 16384 x 16384 channel (268 M fluid cells; population planes 2^28
    elements apart, so plane offsets pass 2^32 elements and bytes): Couette
    flow with a moving hot top wall, a cold bottom wall and a body force,
    5 steps from rest. The flow is uniform along the periodic x direction, so
    each row equals the same row of a 4-wide channel run by the oracle; rows at
    both walls and in the middle are read back with lbm_read_macro_rows."""
    import paper_1510_08224_gb300 as P
    H, K = 16384, 5
    big = lc.couette(H=H, nx=16384, U0=0.05).with_(ax=1e-4)
    small = lc.couette(H=H, nx=4, U0=0.05).with_(ax=1e-4)
    lat = P.Lattice(big, storage=storage)
    lat.step(K)
    o = oracle.OracleLattice(small)
    o.step(K)
    om = o.macro()
    umax = max(np.abs(om[1]).max(), 1e-300)
    tol = {"f64": 1e-12, "f32": 1e-5, "f16": 5e-3}[storage]
    for y0, y1 in ((0, 8), (H // 2 - 2, H // 2 + 2), (H - 6, H + 2)):
        g = lat.macro_rows(y0, y1)
        assert g[0].shape == (y1 - y0, 16384)
        for k, (a, b) in enumerate(zip(g, om)):
            b = b[y0:y1, :1]
            assert np.abs(a - a[:, :1]).max() == 0.0, (k, y0)  # uniform along x
            scale = {0: 1.0, 1: umax, 2: umax, 3: 1.0}[k]
            assert np.abs(a[:, :1] - b).max() <= tol * scale, (k, y0, np.abs(a[:, :1] - b).max())
    lat.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_tall_column_beyond_the_grid_y_limit(storage):
    """A 4-wide, 200,000-row channel: more rows than one launch's grid can
    cover in y (65,535 block rows), so every step kernel walks the rows. The
    whole field after 5 steps from rest equals the oracle's."""
    import paper_1510_08224_gb300 as P
    case = lc.couette(H=200_000, nx=4, U0=0.05).with_(ax=1e-4)
    lat = P.Lattice(case, storage=storage)
    lat.step(5)
    o = oracle.OracleLattice(case)
    o.step(5)
    om = o.macro()
    umax = np.abs(om[1]).max()
    tol = {"f64": 1e-12, "f32": 1e-5, "f16": 5e-3}[storage]
    for k, (a, b) in enumerate(zip(lat.macro(), om)):
        scale = umax if k in (1, 2) else 1.0
        assert np.abs(a - b).max() <= tol * scale, (k, np.abs(a - b).max())
    lat.close()


def test_largest_lattice_fp16_rows_against_oracle():
    """The largest lattice the ABI accepts in FP16 storage: 32768 x 65535 rows,
    ny * pitch = 2,147,450,880 cells, just below the 2^31 limit on cell
    offsets (178 GB on the device with the residual snapshot). Couette flow
    with a body force, 5 steps from rest; rows at both walls and in the middle
    against the oracle's 4-wide channel, as for the 16384 x 16384 channel.
    Skipped where the GPU or the host has too little free memory."""
    import torch
    import paper_1510_08224_gb300 as P
    H, nx, K = 65533, 32768, 5
    big = lc.couette(H=H, nx=nx, U0=0.05).with_(ax=1e-4)
    p, keep = P.make_params(big, "f16")
    need = P.lbm_footprint_bytes(p)
    assert need > 0, P.load().lbm_last_error(None).decode()
    free_dev, _ = torch.cuda.mem_get_info()
    free_host = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    if free_dev < need + (4 << 30) or free_host < (24 << 30):
        pytest.skip(f"needs {need / 2**30:.0f} GiB on the device and 24 GiB on the host")
    lat = P.Lattice(big, storage="f16")
    lat.step(K)
    o = oracle.OracleLattice(lc.couette(H=H, nx=4, U0=0.05).with_(ax=1e-4))
    o.step(K)
    om = o.macro()
    umax = np.abs(om[1]).max()
    for y0, y1 in ((0, 8), (H // 2 - 2, H // 2 + 2), (H - 6, H + 2)):
        g = lat.macro_rows(y0, y1)
        for k, (a, b) in enumerate(zip(g, om)):
            b = b[y0:y1, :1]
            assert np.abs(a - a[:, :1]).max() == 0.0, (k, y0)
            scale = umax if k in (1, 2) else 1.0
            assert np.abs(a[:, :1] - b).max() <= 5e-3 * scale, (k, y0)
    lat.close()
    del lat
    torch.cuda.empty_cache()
