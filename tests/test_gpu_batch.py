"""Batched execution of lattices of uneven size: every member must produce the
same bits as when stepped alone, whatever the mode (one launch per step,
cooperative persistent launches with a grid barrier, CUDA-graph replay), and
whenever lattices join or leave."""
import numpy as np
import pytest

import lbm_cases as lc

pytestmark = pytest.mark.gpu


def _P():
    import paper_1510_08224_gb300 as P
    return P


def _mix():
    return [
        lc.cavity(n=40, Ra=1e4, n_y=33, noise=1e-3),
        lc.rayleigh_benard(nx=300, H=17, Ra=1e5, sigma=1e-2),
        lc.obstacle_channel(nx=133, H=11, frac=0.12, seed=5),
        lc.periodic_box(37, 9, nu=0.02, alpha=0.03, T0=0.2,
                        T_init=0.2 + 0.1 * lc.uniform01(4, 333).reshape(9, 37)),
        lc.cavity(n=130, Ra=1e5, noise=1e-3),
        lc.cavity_nee(n=45, Ra=1e4, noise=1e-3),  # node-based walls: the fused kind adds their pass
    ]


def _alone(P, case, storage, nsteps, seed):
    lat = P.Lattice(case, storage=storage)
    f0, g0 = lc.random_state(case, seed=seed)
    lat.set_populations(f0, g0)
    lat.step(nsteps)
    return lat.populations()


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("mode", [(1, 0, 1, "fused"), (1, 4, 4, "fused"), (3, 0, 16, "persistent"),
                                  (3, 6, 3, "persistent"), (16, 0, 1, "persistent"), (8, 16, 5, "persistent"),
                                  (1, 0, 4, "concurrent"), (1, 4, 4, "concurrent"),
                                  (1, 4, 1, "concurrent", ("vec4w", 1)), (1, 0, 1, "concurrent", ("vec4", 4)),
                                  (1, 4, 1, "concurrent", ("scalar", 0))])
def test_batch_equals_alone(storage, mode):
    """Every kind, and the concurrent kind with a member kernel set for all
    members (VEC4W, VEC4 at 8 blocks/SM, SCALAR) instead of their own. The
    persistent modes run 3, 16 and 8 steps per launch (as many grid barriers
    in one launch) with 1-16 row segments per unit."""
    P = _P()
    cases = _mix()
    total = 11
    ref = [_alone(P, c, storage, total, 30 + i) for i, c in enumerate(cases)]
    b = P.Batch()
    b.set_mode(*mode[:2])
    b.set_config(-1, mode[2])
    b.set_kind(mode[3])
    if len(mode) > 4:
        b.set_member_kernel(*mode[4])
        assert b.get_member_kernel() == mode[4]
    lats = []
    for i, c in enumerate(cases):
        lat = P.Lattice(c, storage=storage)
        f0, g0 = lc.random_state(c, seed=30 + i)
        lat.set_populations(f0, g0)
        lats.append(lat)
    # lattice 0 takes 3 steps alone before joining; the others join at once
    lats[0].step(3)
    for lat in lats[1:]:
        b.add(lat)
    b.step(2)
    b.add(lats[0])
    b.step(total - 3)  # lattice 0: 3 + 8 = 11 steps; the others: 2 + 8 = 10
    b.remove(lats[1])
    b.step(0)
    lats[1].step(1)    # lattice 1 leaves and takes its 11th step alone
    b.step(1)          # lattice 0 reaches 12, lattices 2-4 reach 11
    b.sync()
    for i, lat in enumerate(lats):
        want_steps = 12 if i == 0 else 11
        assert lat.info()["steps"] == want_steps
        if i == 0:
            ref0 = _alone(P, cases[0], storage, 12, 30)
            f, g = lat.populations()
            assert np.array_equal(f, ref0[0]) and np.array_equal(g, ref0[1])
            continue
        f, g = lat.populations()
        assert np.array_equal(f, ref[i][0]) and np.array_equal(g, ref[i][1]), i
    b.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_tuner_keeps_state_and_picks_a_config(storage):
    P = _P()
    cases = _mix()
    b = P.Batch()
    lats = [P.Lattice(c, storage=storage) for c in cases]
    for lat in lats:
        b.add(lat)
    b.step(5)
    b.sync()
    before = [lat.populations() for lat in lats]
    kind, best, ms = b.tune(trial_steps=4)
    assert kind in ("fused", "persistent", "concurrent")
    if kind == "concurrent":
        # -1: the members' own kernels; 0-4 VEC4 at config c; 5-9 VEC4W at config c - 5
        want = ("auto", 0) if best == -1 else ("vec4" if best < 5 else "vec4w", best % 5)
        assert -1 <= best <= 9 and b.get_member_kernel() == want
    else:
        assert 0 <= best <= (9 if kind == "fused" else 4)
    assert all(m > 0 for m in ms.values()) and len(ms) == 31
    # the mix holds a lattice with node-based walls: the persistent kernel cannot take it
    assert all(np.isinf(ms[f"persistent_cfg{c}"]) and np.isinf(ms[f"persistent_u2_cfg{c}"]) for c in range(5))
    assert kind != "persistent"
    assert b.get_mode()[0] == kind
    after = [lat.populations() for lat in lats]
    for (f0, g0), (f1, g1) in zip(before, after):
        assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    b.step(4)
    b.sync()
    for c, lat in zip(cases, lats):
        ref = P.Lattice(c, storage=storage)
        ref.step(9)
        f, g = lat.populations()
        fr, gr = ref.populations()
        assert np.array_equal(f, fr) and np.array_equal(g, gr)
    if kind != "concurrent":
        assert b.info()["config"] == best


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_tuner_times_every_kind_and_keeps_state(storage):
    """Without node-based walls every candidate runs, the persistent kernel's
    trials included (one launch of 32 recomputed steps, 31 grid barriers); the
    state is unchanged and the chosen kind then steps bit-identically."""
    P = _P()
    cases = _mix()[:5]
    b = P.Batch()
    lats = [P.Lattice(c, storage=storage) for c in cases]
    for lat in lats:
        b.add(lat)
    b.step(3)
    b.sync()
    before = [lat.populations() for lat in lats]
    kind, best, ms = b.tune(trial_steps=64)
    b.sync()
    assert all(np.isfinite(m) and m > 0 for m in ms.values()), ms
    after = [lat.populations() for lat in lats]
    for (f0, g0), (f1, g1) in zip(before, after):
        assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    for k in ("fused", "persistent", "concurrent"):
        b.set_kind(k)
        b.step(2)
    b.sync()
    for i, (c, lat) in enumerate(zip(cases, lats)):
        ref = P.Lattice(c, storage=storage)
        ref.step(9)
        f, g = lat.populations()
        fr, gr = ref.populations()
        assert np.array_equal(f, fr) and np.array_equal(g, gr), i
    b.close()


@pytest.mark.parametrize("graph_steps", [0, 4])
def test_batch_of_more_than_64_members(graph_steps):
    """70 small cavities of uneven size: the per-step fused kernel runs as two
    launches (64 + 6 members) and each member still gets its bits alone."""
    P = _P()
    cases = [lc.cavity(n=6 + (k % 13), Ra=1e4, seed=k, noise=1e-3) for k in range(70)]
    b = P.Batch()
    b.set_kind("fused")
    b.set_mode(1, graph_steps)
    lats = [P.Lattice(c, storage="f32", stream=b.stream) for c in cases]
    for lat in lats:
        b.add(lat)
    b.step(8)
    b.sync()
    for c, lat in zip(cases, lats):
        ref = P.Lattice(c, storage="f32")
        ref.step(8)
        f, g = lat.populations()
        fr, gr = ref.populations()
        assert np.array_equal(f, fr) and np.array_equal(g, gr)
    b.close()


def test_batched_lattice_rejects_lbm_step_and_fp64():
    P = _P()
    b = P.Batch()
    lat = P.Lattice(lc.couette(H=4, nx=3), storage="f32")
    b.add(lat)
    with pytest.raises(P.LBMError):
        lat.step(1)
    with pytest.raises(P.LBMError):
        b.add(P.Lattice(lc.couette(H=4, nx=3), storage="f64"))
    with pytest.raises(P.LBMError):
        b.add(P.Lattice(lc.couette(H=4, nx=3), storage="f16"))  # storage mix
    b.remove(lat)
    lat.step(1)


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("config,graph_steps", [(5, 0), (6, 4), (8, 4), (9, 0)])
def test_fused_per_warp_configs_equal_alone(storage, config, graph_steps):
    """The FUSED kind's configs 5-9 (one 128-cell row segment per warp, each warp
    finding its own member): every member of the uneven mix, node-based walls
    included, produces the bits it produces alone."""
    P = _P()
    cases = _mix()
    b = P.Batch()
    b.set_mode(1, graph_steps)
    b.set_config(config, 1)
    lats = []
    for i, c in enumerate(cases):
        lat = P.Lattice(c, storage=storage)
        lat.set_populations(*lc.random_state(c, seed=80 + i))
        b.add(lat)
        lats.append(lat)
    b.step(9)
    b.sync()
    assert b.info()["config"] == config
    for i, (c, lat) in enumerate(zip(cases, lats)):
        f, g = lat.populations()
        fr, gr = _alone(P, c, storage, 9, 80 + i)
        assert np.array_equal(f, fr) and np.array_equal(g, gr), i
    with pytest.raises(P.LBMError):
        b.set_config(10, 1)
    b.close()


def test_member_kernel_choices_and_refusals():
    """The concurrent kind's member kernel: invalid choices are refused and
    leave it unchanged; a member's own kernel change after the batch's graph
    was captured is taken up (a new capture) with the same bits."""
    P = _P()
    cases = _mix()[:3]
    b = P.Batch()
    lats = []
    for i, c in enumerate(cases):
        lat = P.Lattice(c, storage="f32")
        lat.set_populations(*lc.random_state(c, seed=60 + i))
        b.add(lat)
        lats.append(lat)
    assert b.get_member_kernel() == ("auto", 0)
    for bad in (("tma", 0), ("vec8", 0), ("vec4", 5), ("vec4w", -1), ("auto", 1), ("scalar", 1)):
        with pytest.raises(P.LBMError):
            b.set_member_kernel(*bad)
    assert b.get_member_kernel() == ("auto", 0)
    b.set_kind("concurrent")
    b.set_mode(1, 4)
    b.step(4)                          # captures the graph with the members' AUTO kernels
    lats[0].set_step_kernel("scalar")  # changes what the graph holds
    lats[1].set_step_kernel("vec4w", 2)
    b.step(8)
    b.sync()
    for i, (c, lat) in enumerate(zip(cases, lats)):
        f, g = lat.populations()
        fr, gr = _alone(P, c, "f32", 12, 60 + i)
        assert np.array_equal(f, fr) and np.array_equal(g, gr), i
    b.close()


def test_persistent_barrier_timeout_is_reported_and_recoverable():
    """The failure path of the cooperative persistent kernel, without a fault:
    the test hook makes its grid barrier wait for an arrival that never comes,
    the bounded wait (about 2 s) expires, lbm_batch_sync reports LBM_ETIMEOUT,
    and after the hook is cleared the batch works again, bit for bit."""
    import time
    P = _P()
    cases = _mix()[:5]  # no node-based walls: those force one launch per step
    b = P.Batch()
    lats = [P.Lattice(c, storage="f32", stream=b.stream) for c in cases]
    for lat in lats:
        b.add(lat)
    b.set_kind("persistent")
    b.set_mode(4, 0)
    b.debug_barrier_extra(1)
    t0 = time.perf_counter()
    b.step(4)
    with pytest.raises(P.LBMError) as e:
        b.sync()
    assert e.value.status == 5  # LBM_ETIMEOUT
    assert time.perf_counter() - t0 < 60
    with pytest.raises(P.LBMError):
        b.debug_barrier_extra(2)
    b.debug_barrier_extra(0)
    for i, (c, lat) in enumerate(zip(cases, lats)):
        f0, g0 = lc.random_state(c, seed=70 + i)
        lat.set_populations(f0, g0)
    b.step(8)
    b.sync()
    for i, (c, lat) in enumerate(zip(cases, lats)):
        f, g = lat.populations()
        fr, gr = _alone(P, c, "f32", 8, 70 + i)
        assert np.array_equal(f, fr) and np.array_equal(g, gr), i
    b.close()
