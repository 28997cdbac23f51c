"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/*.h declares, and validates parameters."""
import ctypes as C
import glob
import os
import re

import pytest

import lbm_cases as lc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(lbm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    d = _declared()
    for n in ("lbm_create", "lbm_step", "lbm_read_macro", "lbm_nusselt", "lbm_residual", "lbm_destroy"):
        assert n in d


def test_library_exports_every_declared_symbol():
    import paper_1510_08224_gb300 as P
    L = P.load()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(P.EXPORTED) == _declared()


def test_step_kernel_counts_on_host():
    """Every variant's config count per storage (a host-only call): FP64 has the
    scalar kernel only; VEC4 and its per-warp form VEC4W five configs each."""
    import paper_1510_08224_gb300 as P
    assert P.step_kernel_count("f64", "scalar") == 1
    for v in ("vec4", "vec4w", "vec8", "tma"):
        assert P.step_kernel_count("f64", v) == 0
    for st in ("f32", "f16"):
        assert P.step_kernel_count(st, "vec4") == 5 and P.step_kernel_count(st, "vec4w") == 5
    assert P.step_kernel_count("f32", "vec8") == 0 and P.step_kernel_count("f16", "vec8") == 2
    assert ("vec4w", 4) in P.step_kernels("f16") and ("vec4w", 0) in P.step_kernels("f32")


def test_footprint_and_validation_on_host():
    import paper_1510_08224_gb300 as P
    L = P.load()
    case = lc.rayleigh_benard(nx=4096, H=2048, sigma=0.0)
    sizes = {}
    for st in ("f64", "f32", "f16"):
        p, keep = P.make_params(case, st)
        sizes[st] = L.lbm_footprint_bytes(C.byref(p))
    # two buffers of 14 planes dominate: bytes scale with the element size
    assert sizes["f16"] < sizes["f32"] < sizes["f64"]
    plane = case.ny * 4096
    assert sizes["f32"] >= 2 * 14 * 4 * plane
    for b in (case.with_(nu=-0.1), case.with_(s_e=2.0), case.with_(varpi=1.0)):
        p, keep = P.make_params(b, "f32")
        assert L.lbm_footprint_bytes(C.byref(p)) == 0
        assert L.lbm_last_error(None)
        assert L.lbm_validate(C.byref(p)) == 1
    # flag maps: lbm_validate checks them (lbm_footprint_bytes only where the size depends on them)
    fl = case.flags.copy(); fl[0, 0] = 7
    for b in (case.with_(periodic_x=False), case.with_(flags=fl)):
        p, keep = P.make_params(b, "f32")
        assert L.lbm_validate(C.byref(p)) == 1 and L.lbm_last_error(None)
        assert L.lbm_footprint_bytes(C.byref(p)) == sizes["f32"]
    p, keep = P.make_params(case, "f32")
    assert L.lbm_validate(C.byref(p)) == 0


def test_create_rejects_invalid_params_without_touching_the_gpu():
    import paper_1510_08224_gb300 as P
    L = P.load()
    p, keep = P.make_params(lc.couette(H=4, nx=3).with_(alpha=0.0), "f32")
    h = C.c_void_p()
    st = L.lbm_create(C.byref(p), None, None, 0, C.byref(h))
    assert st == 1 and not h.value
    assert b"alpha" in L.lbm_last_error(None)


def test_null_handles_are_errors():
    import paper_1510_08224_gb300 as P
    L = P.load()
    assert L.lbm_step(None, 1) == 1
    assert L.lbm_sync(None) == 1
    L.lbm_destroy(None)


def test_validation_edge_cases_on_host():
    """Parameter and flag-map checks that need no GPU (lbm_validate runs the
    checks of lbm_create on the host): size limit, degenerate lattices, the
    D2Q9 temperature model's and BGK's parameters, and the first invalid cell
    reported in row-major order whatever the number of scanning threads."""
    import paper_1510_08224_gb300 as P
    L = P.load()

    def footprint(case, st="f32"):
        """lbm_footprint_bytes if lbm_validate accepts the case, else 0 (and
        the message)."""
        p, keep = P.make_params(case, st)
        if L.lbm_validate(C.byref(p)) != 0:
            return 0, L.lbm_last_error(None).decode()
        return L.lbm_footprint_bytes(C.byref(p)), L.lbm_last_error(None).decode()

    # ny * pitch must stay below 2^31: rejected before the flag map is read
    small = lc.periodic_box(4, 4)
    p, keep = P.make_params(small, "f32")
    p.nx, p.ny = 65536, 40000
    assert L.lbm_footprint_bytes(C.byref(p)) == 0
    assert "too large" in L.lbm_last_error(None).decode()
    # an empty lattice is rejected
    p.nx, p.ny = 0, 4
    assert L.lbm_footprint_bytes(C.byref(p)) == 0 and "nx and ny" in L.lbm_last_error(None).decode()
    # the smallest lattices: one periodic cell, one periodic column
    assert footprint(lc.periodic_box(1, 1))[0] > 0
    assert footprint(lc.periodic_box(1, 7))[0] > 0
    # D2Q9 temperature model and BGK switch
    q9 = lc.with_d2q9_temperature(lc.couette(H=6, nx=5))
    n5, _ = footprint(lc.couette(H=6, nx=5))
    n9, _ = footprint(q9)
    assert n9 > n5  # four more planes per buffer
    assert footprint(q9.with_(zeta_q=2.0))[0] == 0
    assert footprint(q9.with_(thermal_q=7))[0] == 0
    assert footprint(lc.with_bgk(q9))[0] == n9
    assert footprint(q9.with_(collision=3))[0] == 0
    # a boundary node of an extrapolated wall with no fluid neighbour
    nee = lc.cavity_nee(n=8)
    fl = nee.flags.copy(); fl[1:4, 1:4] = 1  # bury the corner node (0, 0) under wall cells
    n, msg = footprint(nee.with_(flags=fl))
    assert n == 0 and "boundary node" in msg
    # the first invalid cell in row-major order, with errors in many row bands
    big = lc.periodic_box(512, 1024)
    fl = big.flags.copy()
    fl[900, 17] = 5
    fl[300, 400] = 9
    fl[301, 2] = 6
    n, msg = footprint(big.with_(flags=fl))
    assert n == 0 and msg == "cell (400, 300) has wall id 9 > n_walls", msg


def test_flag_map_errors_each_named_at_their_cell():
    """Each kind of invalid flag map is rejected with the cell that makes it
    invalid, on lattices large enough to be scanned by several host threads:
    a fluid cell on a non-periodic edge, a fluid cell whose eight neighbours
    are all bounce-back walls, a wall id above n_walls seen first as a
    neighbour of valid rows."""
    import paper_1510_08224_gb300 as P
    L = P.load()

    def footprint(case):
        p, keep = P.make_params(case, "f32")
        if L.lbm_validate(C.byref(p)) != 0:
            return 0, L.lbm_last_error(None).decode()
        return L.lbm_footprint_bytes(C.byref(p)), L.lbm_last_error(None).decode()

    big = lc.periodic_box(600, 900)
    assert footprint(big)[0] > 0
    # a non-periodic y edge: the first fluid cell of row 0 pulls from outside
    n, msg = footprint(big.with_(periodic_y=False))
    assert n == 0 and msg.startswith("fluid cell (0, 0) touches a non-periodic edge"), msg
    # a channel with walls on both sides is valid
    ch = lc.couette(H=900, nx=600)
    assert footprint(ch)[0] > 0
    # an isolated fluid cell inside a block of bounce-back cells
    fl = ch.flags.copy()
    fl[700:703, 100:103] = 1
    fl[701, 101] = 0
    n, msg = footprint(ch.with_(flags=fl))
    assert n == 0 and msg == "fluid cell (101, 701) has no fluid neighbour", msg
    # a bad id in row 451 is the neighbour of fluid cells in rows 450 and 452
    fl = ch.flags.copy()
    fl[451, 333] = 7
    n, msg = footprint(ch.with_(flags=fl))
    assert n == 0 and msg == "cell (333, 451) has wall id 7 > n_walls", msg
    # removing the top wall row leaves fluid cells on a non-periodic edge
    fl = ch.flags.copy()
    fl[-1, :] = 0
    n, msg = footprint(ch.with_(flags=fl))
    assert n == 0 and msg.startswith(f"fluid cell (0, {ch.ny - 1}) touches a non-periodic edge"), msg
