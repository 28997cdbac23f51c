"""Batched execution against the FP64 oracle.

Every batch kind (the fused per-step kernel, launched directly or replayed
from a CUDA graph; the cooperative persistent kernel with its grid barrier;
the concurrent kind of per-member kernels) advances a mix of lattices of
uneven size, rates and boundary layouts: two differentially heated cavities
(Sec. 3.4) of different size and Rayleigh number, two Rayleigh-Benard cells
periodic in x (one wider than a block row of 512 cells, with a ragged tail),
and a periodic channel with scattered solid cells and a moving heated lid.
Each member is compared element by element with the oracle advanced from
the same state (Eqs. 8-9, 24-25), within the rounding of the storage format:
one step and four steps (a graph replay; two grid barriers inside one
persistent launch) from the same quantised off-equilibrium state, and 400 steps from the
members' own initial states.
"""
import numpy as np
import pytest

import lbm_cases as lc
import oracle

pytestmark = pytest.mark.gpu

# |gpu - oracle| per step, relative to the deviation scale of the state (the
# single-lattice bound of tests/test_gpu_parity.py)
ONE_STEP_TOL = {"f32": 2e-6, "f16": 2e-3}

# (steps_per_launch, graph_steps, rows_per_unit, kind)
MODES = {
    "fused_launch": (1, 0, 1, "fused"),
    "fused_graph": (1, 4, 1, "fused"),
    "persistent_rows1": (3, 0, 1, "persistent"),
    "persistent_rows3": (3, 0, 3, "persistent"),
    "concurrent_graph": (1, 4, 1, "concurrent"),
}


def _P():
    import paper_1510_08224_gb300 as P
    return P


def _mix():
    return [
        lc.cavity(n=40, Ra=1e4, n_y=33, noise=1e-3),
        lc.rayleigh_benard(nx=300, H=17, Ra=1e5, sigma=1e-2),
        lc.rayleigh_benard(nx=700, H=9, Ra=3e4, sigma=1e-2, seed=3),
        lc.obstacle_channel(nx=133, H=11, frac=0.12, seed=5),
        lc.cavity(n=130, Ra=1e5, noise=1e-3),
    ]


def _batch(P, mode):
    spl, graph, rows, kind = mode
    b = P.Batch()
    b.set_mode(spl, graph)
    b.set_config(-1, rows)
    b.set_kind(kind)
    return b


def _dev_scale(case, f, g, keep=None):
    """Largest deviation from the rest state over the cells that carry
    populations (fluid cells, and the boundary nodes of node-based walls)."""
    w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    wT = np.array([1 - case.varpi] + [case.varpi / 4] * 4)[:, None, None]
    keep = (case.flags == 0) if keep is None else keep
    return np.abs(f - w9)[:, keep].max(), np.abs(g - wT * case.T0)[:, keep].max()


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("nsteps", [1, 4])
def test_batch_from_quantised_state_matches_oracle(storage, mode, nsteps):
    """Each member starts from a seeded off-equilibrium state, read back after
    the storage quantised it; the batch advances nsteps (4 steps: one graph
    replay of 4 steps for the graph modes; for the persistent kind one launch of
    3 steps, with two grid barriers, and one of 1) and every population of
    every member is compared with the oracle's."""
    P = _P()
    cases = _mix()
    b = _batch(P, MODES[mode])
    lats, start = [], []
    for i, c in enumerate(cases):
        lat = P.Lattice(c, storage=storage)
        f0, g0 = lc.random_state(c, seed=40 + i)
        lat.set_populations(f0, g0)
        start.append(lat.populations())
        lats.append(lat)
        b.add(lat)
    b.step(nsteps)
    b.sync()
    for i, (c, lat) in enumerate(zip(cases, lats)):
        o = oracle.OracleLattice(c)
        o.set_populations(*start[i])
        o.step(nsteps)
        fo, go = o.populations()
        fg, gg = lat.populations()
        sf, sg = _dev_scale(c, fo, go)
        tol = nsteps * ONE_STEP_TOL[storage]
        ef, eg = np.abs(fg - fo).max() / sf, np.abs(gg - go).max() / sg
        assert ef <= tol and eg <= tol, (i, c.name, ef, eg)
        assert lat.info()["steps"] == nsteps
    b.close()


# Max-norm errors after 400 steps from the members' initial states: u relative
# to the problem's velocity scale (u_c = Ma c_s for the convection cells, the
# lid speed for the channel; a member's own max |u| is no scale while its flow
# is still growing from noise), T relative to its temperature difference (the
# channel: lid to bottom, 1). Bounds: the single-lattice many-step statements
# (FP32 about 1e-7 per step at most, FP16 the cavity's measured 1.2e-2 / 7e-3
# over 4000 steps), with margin.
MANY_TOL = {"f32": {"u": 1e-5, "T": 1e-5}, "f16": {"u": 5e-2, "T": 2e-2}}


def _u_scale(case):
    if "Ma" in case.meta:
        return case.meta["Ma"] * np.sqrt(1.0 / 3.0)
    return max(np.hypot(w.ux, w.uy) for w in case.walls)


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("mode", ["fused_graph", "persistent_rows1", "concurrent_graph"])
def test_batch_many_steps_against_oracle(storage, mode):
    P = _P()
    cases = _mix()
    b = _batch(P, MODES[mode])
    lats = [P.Lattice(c, storage=storage) for c in cases]
    for lat in lats:
        b.add(lat)
    K = 400
    b.step(K)
    b.sync()
    for i, (c, lat) in enumerate(zip(cases, lats)):
        o = oracle.OracleLattice(c)
        o.step(K)
        _, uxo, uyo, To = o.macro()
        _, ux, uy, T = lat.macro()
        us = _u_scale(c)
        dT = getattr(c, "delta_T", 1.0) or 1.0
        eu = max(np.abs(ux - uxo).max(), np.abs(uy - uyo).max()) / us
        eT = np.abs(T - To).max() / dT
        print(f"{mode} {storage} member {i} ({c.name} {c.nx}x{c.ny}): u {eu:.2e} of u scale {us:.3e} "
              f"(max|u| {max(np.abs(uxo).max(), np.abs(uyo).max()):.2e}), T {eT:.2e}")
        assert eu <= MANY_TOL[storage]["u"] and eT <= MANY_TOL[storage]["T"], (i, eu, eT)
    b.close()


def test_batch_with_node_walls_against_oracle():
    """A member with node-based walls (non-equilibrium extrapolation, the
    paper's walls) in a fused batch: its boundary-node pass runs after the
    fused kernel each step; 3 steps from a quantised state against the oracle."""
    P = _P()
    cases = [lc.cavity_nee(n=45, Ra=1e4, noise=1e-3), lc.cavity(n=40, Ra=1e4, n_y=33, noise=1e-3)]
    b = _batch(P, MODES["fused_graph"])
    lats, start = [], []
    for i, c in enumerate(cases):
        lat = P.Lattice(c, storage="f32")
        f0, g0 = lc.random_state(c, seed=60 + i)
        lat.set_populations(f0, g0)
        start.append(lat.populations())
        lats.append(lat)
        b.add(lat)
    b.step(3)
    b.sync()
    for i, (c, lat) in enumerate(zip(cases, lats)):
        o = oracle.OracleLattice(c)
        o.set_populations(*start[i])
        o.step(3)
        fo, go = o.populations()
        fg, gg = lat.populations()
        keep = np.ones(c.flags.shape, bool) if c.name.endswith("nee") else None  # boundary nodes carry populations
        sf, sg = _dev_scale(c, fo, go, keep)
        assert np.abs(fg - fo).max() <= 3 * ONE_STEP_TOL["f32"] * sf, i
        assert np.abs(gg - go).max() <= 3 * ONE_STEP_TOL["f32"] * sg, i
    b.close()
