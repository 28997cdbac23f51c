"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 storage: element-by-element on populations and fields, max-norm relative
error <= 1e-12 (also after 10^4 steps). FP32/FP16-shifted storage: one step
from the same (quantised) state against the oracle within the rounding of the
storage format, and the accumulated max-norm error in u and T after many steps
is checked against a stated bound.
"""
import numpy as np
import pytest

import lbm_cases as lc
import oracle

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _P():
    import paper_1510_08224_gb300 as P
    return P


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _cases_small():
    return [
        lc.periodic_box(7, 5, nu=0.03, alpha=0.04, g_beta=2e-3, T0=0.5,
                        kinetic=dict(s_e=1.3, s_q=1.1, s_eps=1.5, zeta_e=1.2, zeta_nu=0.9), ax=1e-5),
        lc.couette(H=9, nx=5, U0=0.05),
        lc.porous_couette(H=16, nx=3),
        lc.cavity(n=20, Ra=1e4, n_y=13, noise=1e-3),
        lc.rayleigh_benard(nx=133, H=7, Ra=1e5, sigma=1e-2),  # two x blocks plus a ragged tail
        lc.poiseuille(H=11, nx=1, ax=1e-5),                   # nx = 1: periodic self-neighbour
        lc.obstacle_channel(nx=261, H=9, frac=0.15, seed=4),  # scattered solid cells, moving lid
        lc.periodic_box(6, 9, nu=0.02, alpha=0.03, T0=0.2,
                        T_init=0.2 + 0.1 * lc.uniform01(9, 54).reshape(9, 6)),  # periodic in x and y
        lc.cavity_nee(n=19, Ra=1e4, noise=1e-3),                 # node-based walls on all four sides
        lc.porous_couette_nee(H=13, nx=5, Re=10, s_nu=0.8),       # node-based moving, injecting walls
    ]


N_SMALL = 10


@pytest.mark.parametrize("idx", range(N_SMALL))
@pytest.mark.parametrize("nsteps", [0, 1, 2, 10])
def test_fp64_populations_match_oracle(idx, nsteps):
    P = _P()
    case = _cases_small()[idx]
    g = P.Lattice(case, storage="f64")
    o = oracle.OracleLattice(case)
    if idx in (0, 6, 7, 8):  # start off-equilibrium
        f0, g0 = lc.random_state(case, seed=11)
        g.set_populations(f0, g0)
        o.set_populations(f0, g0)
    g.step(nsteps)
    o.step(nsteps)
    fg, gg = g.populations()
    fo, go = o.populations()
    assert _rel(fg, fo) <= FP64_TOL
    assert _rel(gg, go) <= FP64_TOL
    for a, b in zip(g.macro(), o.macro()):
        assert np.abs(a - b).max() <= FP64_TOL * max(np.abs(b).max(), 1.0)


def test_fp64_injection_channel_1e4_steps():
    """Porous-plate thermal Couette, 8 x 64 fluid cells, 10^4 steps."""
    P = _P()
    case = lc.porous_couette(H=64, nx=8)
    g = P.Lattice(case, storage="f64")
    o = oracle.OracleLattice(case)
    g.step(10000)
    o.step(10000)
    for a, b in zip(g.macro(), o.macro()):
        assert _rel(a, b) <= FP64_TOL
    fg, gg = g.populations()
    fo, go = o.populations()
    assert _rel(fg, fo) <= FP64_TOL and _rel(gg, go) <= FP64_TOL
    # mass: the injecting and sucking walls balance exactly
    assert abs(fg.sum() - fo.sum()) / fo.sum() < 1e-13


def test_fp64_convective_cavity_1e4_steps():
    P = _P()
    case = lc.cavity(n=32, Ra=1e4, noise=1e-3)
    g = P.Lattice(case, storage="f64")
    o = oracle.OracleLattice(case, threads=4)
    g.step(10000)
    o.step(10000)
    for a, b in zip(g.macro()[1:], o.macro()[1:]):
        assert _rel(a, b) <= FP64_TOL
    for side in (0, 1):
        assert abs(g.nusselt(side) - o.nusselt(side)) <= 1e-11


def _quantised_start(P, case, storage, seed):
    """Load a random state into the GPU lattice and read back what the storage
    format holds, so the oracle starts from exactly the same numbers."""
    g = P.Lattice(case, storage=storage)
    f0, g0 = lc.random_state(case, seed=seed)
    g.set_populations(f0, g0)
    fq, gq = g.populations()
    return g, fq, gq


# one-step bound on |gpu - oracle| relative to the deviation scale of the state
ONE_STEP_TOL = {"f32": 2e-6, "f16": 2e-3}


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("idx", range(N_SMALL))
def test_reduced_precision_one_step(storage, idx):
    P = _P()
    case = _cases_small()[idx]
    g, fq, gq = _quantised_start(P, case, storage, seed=5 + idx)
    o = oracle.OracleLattice(case)
    o.set_populations(fq, gq)
    g.step(1)
    o.step(1)
    fg, gg = g.populations()
    fo, go = o.populations()
    w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    wT = np.array([1 - case.varpi] + [case.varpi / 4] * 4)[:, None, None]
    solid = case.flags != 0
    dev_f = np.where(solid, 0.0, fo - w9)
    dev_g = np.where(solid, 0.0, go - wT * case.T0)
    scale_f, scale_g = np.abs(dev_f).max(), np.abs(dev_g).max()
    assert np.abs(fg - fo).max() <= ONE_STEP_TOL[storage] * scale_f
    assert np.abs(gg - go).max() <= ONE_STEP_TOL[storage] * scale_g


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("idx", range(N_SMALL))
def test_step_variants_agree_bitwise(storage, idx):
    """The scalar, vectorised and TMA-staged step kernels run the same
    arithmetic: five steps from the same state give the same bits."""
    P = _P()
    case = _cases_small()[idx]
    f0, g0 = lc.random_state(case, seed=21 + idx)
    out = {}
    for v in P.step_kernels(storage):
        lat = P.Lattice(case, storage=storage)
        lat.set_step_kernel(*v)
        lat.set_populations(f0, g0)
        lat.step(5)
        out[v] = lat.populations()
        lat.sync()
    ref = out[("scalar", 0)]
    for v, o in out.items():
        assert np.array_equal(o[0], ref[0]) and np.array_equal(o[1], ref[1]), v


def test_fp64_rejects_vector_variants():
    P = _P()
    lat = P.Lattice(lc.couette(H=4, nx=3), storage="f64")
    lat.set_step_kernel("scalar")
    with pytest.raises(P.LBMError):
        lat.set_step_kernel("tma")
    assert P.step_kernel_count("f64", "tma") == 0 and P.step_kernel_count("f32", "tma") == 5
    assert P.step_kernel_count("f32", "vec8") == 0 and P.step_kernel_count("f16", "vec8") == 2
    assert P.step_kernel_count("f64", "vec4w") == 0
    assert P.step_kernel_count("f32", "vec4w") == 5 and P.step_kernel_count("f16", "vec4w") == 5


# Accumulated max-norm error after 4000 steps against the FP64 oracle. FP16
# deviations carry an 11-bit significand, so each step rounds every population
# by up to ~1e-4 of its deviation; the measured error on this case is about
# 1.2e-2 of max|u| and 7e-3 of delta T, bounded here with margin.
MANY_STEP_TOL = {"f32": {"u": 1e-6, "T": 1e-6}, "f16": {"u": 2.5e-2, "T": 1.5e-2}}


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_reduced_precision_cavity_error(storage):
    """Cavity at Ra = 1e4 from rest, 4000 steps: max-norm error in u (relative
    to max |u|) and T (relative to delta T) against the FP64 oracle."""
    P = _P()
    case = lc.cavity(n=32, Ra=1e4, noise=1e-3)
    g = P.Lattice(case, storage=storage)
    o = oracle.OracleLattice(case, threads=4)
    g.step(4000)
    o.step(4000)
    _, uxg, uyg, Tg = g.macro()
    _, uxo, uyo, To = o.macro()
    umax = max(np.abs(uxo).max(), np.abs(uyo).max())
    eu = max(np.abs(uxg - uxo).max(), np.abs(uyg - uyo).max()) / umax
    eT = np.abs(Tg - To).max() / case.delta_T
    print(f"{storage}: max-norm error u {eu:.3e} (of max|u|), T {eT:.3e} (of dT)")
    assert eu <= MANY_STEP_TOL[storage]["u"] and eT <= MANY_STEP_TOL[storage]["T"]


def test_fp16_error_is_the_storage_rounding():
    """The FP16-shifted path's error on the 32 x 32 cavity (Ra = 1e4, 4000
    steps) against the exact FP64 oracle is the error of the oracle itself
    when only its stored deviations are rounded to binary16 after every step
    (FP64 arithmetic otherwise): the same size within a factor 1.5. So the
    FP16 floor comes from the 11-bit significand of the stored state, not from
    the kernels' FP32 arithmetic."""
    P = _P()
    case = lc.cavity(n=32, Ra=1e4, noise=1e-3)
    ref = oracle.OracleLattice(case, threads=4)
    ref.step(4000)
    emu = oracle.OracleLattice(case, threads=4)
    emu.set_storage_rounding(16, 1.0)
    emu.step(4000)
    g = P.Lattice(case, storage="f16")
    g.step(4000)
    _, uxo, uyo, To = ref.macro()
    umax = max(np.abs(uxo).max(), np.abs(uyo).max())

    def err(m):
        return (max(np.abs(m[1] - uxo).max(), np.abs(m[2] - uyo).max()) / umax, np.abs(m[3] - To).max())
    eg, ee = err(g.macro()), err(emu.macro())
    print(f"FP16 path: u {eg[0]:.3e}, T {eg[1]:.3e}; oracle with binary16 storage: u {ee[0]:.3e}, T {ee[1]:.3e}")
    for a, b in zip(eg, ee):
        assert b / 1.5 <= a <= 1.5 * b


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_macro_nusselt_residual_match_oracle(storage):
    P = _P()
    case = lc.cavity(n=24, Ra=1e4, noise=1e-3)
    g, fq, gq = _quantised_start(P, case, storage, seed=3)
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
    with pytest.raises(P.LBMError):
        g.nusselt("top")  # adiabatic wall


def _full_size_sampled(storage, seed, nsample=3000, nx=4096):
    """Rayleigh-Benard at the benchmark size (4096 x 2048 fluid cells plus the
    two wall rows), the benchmark's launch configuration: one step from a
    seeded random state, every population of sampled nodes against the
    oracle's single-node update."""
    P = _P()
    case = lc.rayleigh_benard(nx=nx, H=2048, sigma=0.0)
    g, fq, gq = _quantised_start(P, case, storage, seed=seed)
    g.step(1)
    f1, g1 = g.populations()
    o = oracle.OracleLattice(case.with_(T_init=None))
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, case.nx, nsample)
    ys = rng.integers(1, case.ny - 1, nsample)
    # always include the seam of the periodic wrap and the wall rows
    xs[:4] = [0, case.nx - 1, 0, case.nx - 1]
    ys[:4] = [1, 1, case.ny - 2, case.ny - 2]
    fq = np.ascontiguousarray(fq); gq = np.ascontiguousarray(gq)
    ef = eg = 0.0
    sf = sg = 0.0
    for x, y in zip(xs, ys):
        fo, go = o.update_node(fq, gq, int(x), int(y))
        ef = max(ef, np.abs(f1[:, y, x] - fo).max())
        eg = max(eg, np.abs(g1[:, y, x] - go).max())
        sf = max(sf, np.abs(fo - np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)).max())
        sg = max(sg, np.abs(go - np.array([0.5] + [0.125] * 4) * case.T0).max())
    # the rest of the lattice: mass and T are conserved away from the walls' exchange
    return ef, eg, sf, sg


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_full_size_sampled_nodes(storage):
    ef, eg, sf, sg = _full_size_sampled(storage, seed=17)
    if storage == "f64":
        assert ef <= FP64_TOL and eg <= FP64_TOL
    else:
        assert ef <= ONE_STEP_TOL[storage] * sf and eg <= ONE_STEP_TOL[storage] * sg


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_full_size_ragged_width_sampled_nodes(storage):
    """The same at 4000 x 2048, whose rows are not a multiple of 512 cells: the
    AUTO kernel is the per-warp form (VEC4W) in FP32 and the four-cell kernel
    with a partly filled last block per row in FP16."""
    ef, eg, sf, sg = _full_size_sampled(storage, seed=23, nsample=2000, nx=4000)
    assert ef <= ONE_STEP_TOL[storage] * sf and eg <= ONE_STEP_TOL[storage] * sg


def test_library_allocated_memory_and_side_stream():
    import torch
    P = _P()
    case = lc.cavity(n=16, Ra=1e4, noise=1e-3)
    s = torch.cuda.Stream()
    a = P.Lattice(case, storage="f64", stream=s, device_mem="library")
    b = P.Lattice(case, storage="f64")
    a.step(50)
    b.step(50)
    for x, y in zip(a.populations(), b.populations()):
        assert np.array_equal(x, y)
    info = a.info()
    assert info["steps"] == 50 and info["fluid_cells"] == 256


def test_invalid_inputs_are_rejected():
    P = _P()
    c = lc.couette(H=4, nx=3)
    with pytest.raises(P.LBMError):
        P.Lattice(c.with_(periodic_x=False))          # open edge without a frame
    with pytest.raises(P.LBMError):
        P.Lattice(c.with_(nu=-1.0))                   # rate outside (0, 2)
    with pytest.raises(P.LBMError):
        P.Lattice(c.with_(s_q=2.0))
    iso = lc.cavity(n=3, noise=0.0)
    fl = iso.flags.copy(); fl[1:-1, 1:-1] = 1; fl[2, 2] = 0  # a fluid cell with no fluid neighbour
    with pytest.raises(P.LBMError):
        P.Lattice(iso.with_(flags=fl))
    g = P.Lattice(c)
    with pytest.raises(P.LBMError):
        g.step(-1)


def test_caller_memory_too_small():
    import ctypes as C
    import torch
    P = _P()
    L = P.load()
    c = lc.couette(H=4, nx=3)
    p, keep = P.make_params(c, "f32")
    need = L.lbm_footprint_bytes(C.byref(p))
    buf = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    h = C.c_void_p()
    st = L.lbm_create(C.byref(p), None, C.c_void_p(buf.data_ptr()), C.c_size_t(need - 256), C.byref(h))
    assert st == 2 and not h.value  # LBM_ENOMEM


def test_nan_state_is_reported_as_diverged():
    P = _P()
    c = lc.couette(H=4, nx=3)
    g = P.Lattice(c, storage="f64")
    f, t = g.populations()
    f[1, 2, 1] = np.nan
    g.set_populations(f, t)
    g.step(2)
    with pytest.raises(P.LBMError) as e:
        g.residual()
    assert e.value.status == 4  # LBM_EDIVERGED


def test_nee_cavity_nusselt_against_table3_on_gpu():
    """Node-based cavity (the paper's walls), Ra = 1e3, 64 x 64 intervals,
    FP64 storage, run to steady state: Nu within 0.5 % of Table 3 (1.1161)
    and equal to the oracle's value after the same steps."""
    import os
    P = _P()
    row = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "table3_cavity.txt"))[0]
    case = lc.cavity_nee(n=64, Ra=1e3)
    g = P.Lattice(case, storage="f64")
    g.residual()
    for _ in range(200):
        g.step(1000)
        if g.residual() < 1e-9:
            break
    nu = [g.nusselt(s, L=64.0) for s in (0, 1)]
    for v in nu:
        assert abs(v - row[5]) / row[5] < 5e-3
    steps = g.info()["steps"]
    o = oracle.OracleLattice(case, threads=8)
    o.step(steps)
    for side, v in zip((0, 1), nu):
        assert abs(v - o.nusselt(side, L=64.0)) < 1e-10


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_graph_replayed_steps_equal_direct_steps(storage):
    """lbm_step replays runs of 4 steps or more as CUDA graphs of 32 and 4
    steps: 201 steps in one call (a direct step, capture, a direct step to the
    graphs' starting buffer, six 32-step and one 4-step replay, three direct
    steps), and runs of 5, 20, 7 and 33 steps, give the bits of as many
    single-step calls, with halfway and node-based walls, on the default stream
    and on a side stream, for the AUTO kernel and (FP32) the TMA kernel; a call
    on a stream that torch is capturing joins that graph and gives the same
    bits when replayed."""
    import torch
    P = _P()
    cases = [lc.rayleigh_benard(nx=133, H=7, Ra=1e5, sigma=1e-2), lc.cavity_nee(n=19, Ra=1e4, noise=1e-3)]
    for case in cases:
        f0, g0 = lc.random_state(case, seed=5)
        variants = [("auto", 0)] + ([("tma", 1)] if storage == "f32" and case.name != "cavity_nee" else [])
        for v in variants:
            for side in (False, True):
                s = torch.cuda.Stream() if side else None
                a = P.Lattice(case, storage=storage, stream=s)
                b = P.Lattice(case, storage=storage, stream=s)
                for lat in (a, b):
                    lat.set_step_kernel(*v)
                    lat.set_populations(f0, g0)
                a.step(201)
                for _ in range(201):
                    b.step(1)
                fa, ga = a.populations()
                fb, gb = b.populations()
                assert np.array_equal(fa, fb) and np.array_equal(ga, gb), (case.name, v, side)
                for n in (5, 20, 7, 33):
                    a.step(n)
                    for _ in range(n):
                        b.step(1)
                fa, ga = a.populations()
                fb, gb = b.populations()
                assert np.array_equal(fa, fb) and np.array_equal(ga, gb), (case.name, v, side, "short runs")
                a.close()
                b.close()
        # inside a capture on the caller's stream
        s = torch.cuda.Stream()
        a = P.Lattice(case, storage=storage, stream=s)
        b = P.Lattice(case, storage=storage, stream=s)
        a.set_populations(f0, g0)
        b.set_populations(f0, g0)
        a.step(1)
        torch.cuda.synchronize()
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=s):
            a.step(64)
        gr.replay()
        gr.replay()
        torch.cuda.synchronize()
        for _ in range(129):
            b.step(1)
        assert np.array_equal(a.populations()[0], b.populations()[0])
        a.close()
        b.close()


def _pinned(a):
    import torch
    t = torch.empty(a.shape, dtype={np.uint8: torch.uint8, np.float64: torch.float64}[a.dtype.type]).pin_memory()
    t.numpy()[...] = a
    return t


@pytest.mark.parametrize("pinned", [False, True])
def test_create_checks_flag_maps_like_validate(pinned):
    """lbm_create builds the link map and checks the flag map on the GPU where
    every wall is halfway: an invalid map is rejected with exactly the message
    of lbm_validate (the host check), whether the map is page-locked (read in
    place) or pageable (copied); a valid one gives the host's fluid-cell
    count."""
    import ctypes as C
    P = _P()
    L = P.load()
    ch = lc.couette(H=900, nx=600)
    box = lc.periodic_box(512, 1024)
    bad = []
    fl = ch.flags.copy(); fl[700:703, 100:103] = 1; fl[701, 101] = 0
    bad.append(ch.with_(flags=fl))                      # a fluid cell with no fluid neighbour
    fl = ch.flags.copy(); fl[451, 333] = 7
    bad.append(ch.with_(flags=fl))                      # a wall id above n_walls
    fl = ch.flags.copy(); fl[-1, :] = 0
    bad.append(ch.with_(flags=fl))                      # fluid cells on a non-periodic edge
    fl = box.flags.copy(); fl[900, 17] = 5; fl[300, 400] = 9; fl[301, 2] = 6
    bad.append(box.with_(flags=fl))                     # several, the first in row-major order named
    bad.append(box.with_(periodic_y=False))
    keep = []
    for case in bad:
        flags = _pinned(case.flags) if pinned else case.flags
        keep.append(flags)
        c2 = case.with_(flags=flags.numpy() if pinned else flags)
        p, k = P.make_params(c2, "f32")
        assert L.lbm_validate(C.byref(p)) == 1
        want = L.lbm_last_error(None)
        h = C.c_void_p()
        assert L.lbm_create(C.byref(p), None, None, 0, C.byref(h)) == 1 and not h.value
        assert L.lbm_last_error(None) == want, (L.lbm_last_error(None), want)
    for case in (ch, box, lc.obstacle_channel(nx=261, H=9, frac=0.15, seed=4), lc.periodic_box(1, 1)):
        flags = _pinned(case.flags) if pinned else case.flags
        lat = P.Lattice(case.with_(flags=flags.numpy() if pinned else flags), storage="f32")
        assert lat.info()["fluid_cells"] == int((case.flags == 0).sum())
        lat.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_create_reads_page_locked_inputs_in_place(storage):
    """Flags and T_init in page-locked memory are read in place by the GPU,
    pageable ones are copied: the initial state is the same bits either way,
    and a tall lattice (more rows than one launch's grid covers) builds its
    maps across the launch seams."""
    P = _P()
    for case in (lc.rayleigh_benard(nx=300, H=17, Ra=1e5, sigma=1e-2),
                 lc.couette(H=70_000, nx=4, U0=0.05).with_(T_init=0.3 + 0.01 * lc.uniform01(3, 70_002 * 4).reshape(70_002, 4))):
        a = P.Lattice(case, storage=storage)
        fl, Ti = _pinned(case.flags), _pinned(case.T_init)
        b = P.Lattice(case.with_(flags=fl.numpy(), T_init=Ti.numpy()), storage=storage)
        fa, ga = a.populations()
        fb, gb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
        a.step(3)
        b.step(3)
        assert all(np.array_equal(x, y) for x, y in zip(a.populations(), b.populations()))
        o = oracle.OracleLattice(case)
        o.step(3)
        if storage == "f64":
            assert _rel(a.populations()[0], o.populations()[0]) <= FP64_TOL
        a.close()
        b.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_read_macro_into_page_locked_arrays(storage):
    """lbm_read_macro writes page-locked host arrays in place (pageable ones
    through the staging area): the same values either way, any output NULL,
    row bands included."""
    import ctypes as C
    import torch
    P = _P()
    L = P.load()
    case = lc.rayleigh_benard(nx=300, H=70, Ra=1e5, sigma=1e-2)
    lat = P.Lattice(case, storage=storage)
    lat.step(40)
    ref = lat.macro()
    outs = [torch.empty((case.ny, case.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    ptr = [C.cast(o.data_ptr(), C.POINTER(C.c_double)) for o in outs]
    assert L.lbm_read_macro(lat.handle, ptr[0], None, ptr[2], ptr[3]) == 0
    for k in (0, 2, 3):
        assert np.array_equal(outs[k].numpy(), ref[k])
    band = [torch.full((10, case.nx), -1.0, dtype=torch.float64).pin_memory() for _ in range(4)]
    bp = [C.cast(o.data_ptr(), C.POINTER(C.c_double)) for o in band]
    assert L.lbm_read_macro_rows(lat.handle, 30, 40, *bp) == 0
    for k in range(4):
        assert np.array_equal(band[k].numpy(), ref[k][30:40])
    lat.close()
