"""Parity of the CUDA path with the FP64 oracle for the D2Q9 temperature model
of Eqs. 31-33 (thermal_q = 9): the same cases as the D2Q5 parity tests, FP64
element by element (<= 1e-12 relative max-norm, also after 10^4 steps),
FP32/FP16 one step from the same quantised state, and every step kernel
variant bit-identical."""
import numpy as np
import pytest

import lbm_cases as lc
import oracle

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]


def _P():
    import paper_1510_08224_gb300 as P
    return P


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _cases():
    q = lc.with_d2q9_temperature
    return [
        q(lc.periodic_box(7, 5, nu=0.03, alpha=0.04, g_beta=2e-3, T0=0.5,
                          kinetic=dict(s_e=1.3, s_q=1.1, s_eps=1.5, zeta_e=1.2, zeta_nu=0.9), ax=1e-5),
          zeta_q=1.1, zeta_eps=1.3),
        q(lc.couette(H=9, nx=5, U0=0.05)),
        q(lc.porous_couette(H=16, nx=3)),                        # injecting walls: u_w normal to the wall
        q(lc.cavity(n=20, Ra=1e4, n_y=13, noise=1e-3)),
        q(lc.rayleigh_benard(nx=133, H=7, Ra=1e5, sigma=1e-2)),  # two x blocks plus a ragged tail
        q(lc.obstacle_channel(nx=261, H=9, frac=0.15, seed=4)),  # moving lid: the theta terms of the wall rule
        q(lc.cavity_nee(n=19, Ra=1e4, noise=1e-3)),              # node-based walls
        q(lc.porous_couette_nee(H=13, nx=5, Re=10, s_nu=0.8)),
        q(lc.obstacle_channel(nx=37, H=9, frac=0.15, seed=5), theta=0.0),  # Eq. 31 without the second-order terms
    ]


N = 9
RANDOM_START = (0, 3, 5, 6, 8)


@pytest.mark.parametrize("idx", range(N))
@pytest.mark.parametrize("nsteps", [0, 1, 2, 10])
def test_d2q9t_fp64_matches_oracle(idx, nsteps):
    P = _P()
    case = _cases()[idx]
    g = P.Lattice(case, storage="f64")
    o = oracle.OracleLattice(case)
    assert o.tq == 9 and g.tq == 9
    if idx in RANDOM_START:
        f0, g0 = lc.random_state(case, seed=31 + idx)
        assert g0.shape[0] == 9
        g.set_populations(f0, g0)
        o.set_populations(f0, g0)
    g.step(nsteps)
    o.step(nsteps)
    fg, gg = g.populations()
    fo, go = o.populations()
    assert gg.shape == go.shape == (9, case.ny, case.nx)
    assert _rel(fg, fo) <= FP64_TOL
    assert _rel(gg, go) <= FP64_TOL
    for a, b in zip(g.macro(), o.macro()):
        assert np.abs(a - b).max() <= FP64_TOL * max(np.abs(b).max(), 1.0)


def test_d2q9t_fp64_cavity_1e4_steps():
    P = _P()
    case = lc.with_d2q9_temperature(lc.cavity(n=32, Ra=1e4, noise=1e-3))
    g = P.Lattice(case, storage="f64")
    o = oracle.OracleLattice(case, threads=4)
    g.step(10000)
    o.step(10000)
    for a, b in zip(g.macro()[1:], o.macro()[1:]):
        assert _rel(a, b) <= FP64_TOL
    for side in (0, 1):
        assert abs(g.nusselt(side) - o.nusselt(side)) <= 1e-11


ONE_STEP_TOL = {"f32": 2e-6, "f16": 2e-3}


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("idx", range(N))
def test_d2q9t_reduced_precision_one_step(storage, idx):
    P = _P()
    case = _cases()[idx]
    g = P.Lattice(case, storage=storage)
    f0, g0 = lc.random_state(case, seed=41 + idx)
    g.set_populations(f0, g0)
    fq, gq = g.populations()
    o = oracle.OracleLattice(case)
    o.set_populations(fq, gq)
    g.step(1)
    o.step(1)
    fg, gg = g.populations()
    fo, go = o.populations()
    solid = case.flags != 0
    solid = solid & np.array([[w.scheme == lc.HALFWAY for w in case.walls][k - 1] if k else False
                              for k in case.flags.ravel()]).reshape(solid.shape)
    dev_f = np.where(solid, 0.0, fo - W9)
    dev_g = np.where(solid, 0.0, go - W9 * case.T0)
    assert np.abs(fg - fo).max() <= ONE_STEP_TOL[storage] * np.abs(dev_f).max()
    assert np.abs(gg - go).max() <= ONE_STEP_TOL[storage] * np.abs(dev_g).max()


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("idx", range(N))
def test_d2q9t_step_variants_agree_bitwise(storage, idx):
    P = _P()
    case = _cases()[idx]
    f0, g0 = lc.random_state(case, seed=51 + idx)
    out = {}
    variants = [("scalar", 0)] + [(v, c) for v in ("vec4", "vec4w") for c in range(P.step_kernel_count(storage, v))] \
        + [("auto", 0)]
    for v in variants:
        lat = P.Lattice(case, storage=storage)
        lat.set_step_kernel(*v)
        lat.set_populations(f0, g0)
        lat.step(5)
        out[v] = lat.populations()
        lat.sync()
    ref = out[("scalar", 0)]
    for v, o in out.items():
        assert np.array_equal(o[0], ref[0]) and np.array_equal(o[1], ref[1]), v


def test_d2q9t_rejects_tma_vec8_and_batches():
    P = _P()
    case = lc.with_d2q9_temperature(lc.couette(H=6, nx=5))
    lat = P.Lattice(case, storage="f16")
    with pytest.raises(P.LBMError):
        lat.set_step_kernel("tma", 0)
    with pytest.raises(P.LBMError):
        lat.set_step_kernel("vec8", 0)
    b = P.Batch()
    lat2 = P.Lattice(case, storage="f32", stream=b.stream)
    with pytest.raises(P.LBMError):
        b.add(lat2)
    b.close()


def test_d2q9t_rejects_bad_rates():
    P = _P()
    case = lc.with_d2q9_temperature(lc.couette(H=6, nx=5))
    with pytest.raises(P.LBMError):
        P.Lattice(case.with_(zeta_q=2.0))
    with pytest.raises(P.LBMError):
        P.Lattice(case.with_(zeta_eps=0.0))
    with pytest.raises(P.LBMError):
        P.Lattice(case.with_(thermal_q=7))


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_d2q9t_macro_nusselt_residual_match_oracle(storage):
    P = _P()
    case = lc.with_d2q9_temperature(lc.cavity(n=24, Ra=1e4, noise=1e-3))
    g = P.Lattice(case, storage=storage)
    f0, g0 = lc.random_state(case, seed=3)
    g.set_populations(f0, g0)
    fq, gq = g.populations()
    o = oracle.OracleLattice(case)
    o.set_populations(fq, gq)
    tol = {"f64": 1e-12, "f32": 1e-6, "f16": 1e-6}[storage]
    for a, b in zip(g.macro(), o.macro()):
        assert np.abs(a - b).max() <= tol * max(1.0, np.abs(b).max())
    for side in (0, 1):
        assert abs(g.nusselt(side) - o.nusselt(side)) <= 50 * tol * abs(o.nusselt(side)) + 1e-12
    assert np.isinf(g.residual()) and np.isinf(o.residual())
    g.step(7)
    o.step(7)
    rg, ro = g.residual(), o.residual()
    rtol = {"f64": 1e-10, "f32": 1e-3, "f16": 1e-2}[storage]
    assert abs(rg - ro) <= rtol * ro


def test_d2q9t_cavity_nusselt_close_to_d2q5():
    """Both temperature models solve the same problem: at steady state
    (Ra = 1e3, 48 x 48 cells, FP64) their mean Nusselt numbers agree within
    the discretisation error (1 %)."""
    P = _P()
    base = lc.cavity(n=48, Ra=1e3)
    nus = []
    for case in (base, lc.with_d2q9_temperature(base)):
        g = P.Lattice(case, storage="f64")
        g.residual()
        for _ in range(100):
            g.step(1000)
            if g.residual() < 1e-9:
                break
        nus.append(g.nusselt(0))
    assert abs(nus[0] - nus[1]) / nus[0] < 1e-2


def _full_size_sampled(case, storage, seed, nsample=2000):
    """Rayleigh-Benard at the benchmark size (4096 x 2048 fluid cells), AUTO step
    kernel: one step from a seeded random state, every population of sampled
    nodes (the periodic seam and the wall rows included) against the oracle's
    single-node update. Returns (max error f, max error g, scale f, scale g)."""
    P = _P()
    g = P.Lattice(case, storage=storage)
    f0, g0 = lc.random_state(case, seed=seed)
    g.set_populations(f0, g0)
    fq, gq = g.populations()
    g.step(1)
    f1, g1 = g.populations()
    o = oracle.OracleLattice(case.with_(T_init=None))
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, case.nx, nsample)
    ys = rng.integers(1, case.ny - 1, nsample)
    xs[:4] = [0, case.nx - 1, 0, case.nx - 1]
    ys[:4] = [1, 1, case.ny - 2, case.ny - 2]
    fq = np.ascontiguousarray(fq); gq = np.ascontiguousarray(gq)
    wT = W9[:, 0, 0] if case.thermal_q == 9 else np.array([0.5, 0.125, 0.125, 0.125, 0.125])
    ef = eg = sf = sg = 0.0
    for x, y in zip(xs, ys):
        fo, go = o.update_node(fq, gq, int(x), int(y))
        ef = max(ef, np.abs(f1[:, y, x] - fo).max())
        eg = max(eg, np.abs(g1[:, y, x] - go).max())
        sf = max(sf, np.abs(fo - W9[:, 0, 0]).max())
        sg = max(sg, np.abs(go - wT * case.T0).max())
    return ef, eg, sf, sg


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_d2q9t_full_size_sampled_nodes(storage):
    case = lc.with_d2q9_temperature(lc.rayleigh_benard(nx=4096, H=2048, sigma=0.0))
    ef, eg, sf, sg = _full_size_sampled(case, storage, seed=23)
    if storage == "f64":
        assert ef <= FP64_TOL * max(sf, 1.0) and eg <= FP64_TOL * max(sg, 1.0)
    else:
        assert ef <= ONE_STEP_TOL[storage] * sf and eg <= ONE_STEP_TOL[storage] * sg


# Accumulated max-norm error after 4000 steps against the FP64 oracle (cavity
# 32 x 32, Ra = 1e4, from rest): measured FP32 u 3.0e-7 (of max |u|), T 1.9e-7
# (of delta T); FP16 u 3.8e-3, T 1.2e-3; bounded with margin.
D2Q9T_MANY_STEP_TOL = {"f32": {"u": 1e-6, "T": 1e-6}, "f16": {"u": 1.5e-2, "T": 5e-3}}


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_d2q9t_reduced_precision_cavity_error(storage):
    P = _P()
    case = lc.with_d2q9_temperature(lc.cavity(n=32, Ra=1e4, noise=1e-3))
    g = P.Lattice(case, storage=storage)
    o = oracle.OracleLattice(case, threads=4)
    g.step(4000)
    o.step(4000)
    _, uxg, uyg, Tg = g.macro()
    _, uxo, uyo, To = o.macro()
    umax = max(np.abs(uxo).max(), np.abs(uyo).max())
    eu = max(np.abs(uxg - uxo).max(), np.abs(uyg - uyo).max()) / umax
    eT = np.abs(Tg - To).max() / case.delta_T
    print(f"D2Q9 T {storage}: max-norm error u {eu:.3e} (of max|u|), T {eT:.3e} (of dT)")
    assert eu <= D2Q9T_MANY_STEP_TOL[storage]["u"] and eT <= D2Q9T_MANY_STEP_TOL[storage]["T"]
