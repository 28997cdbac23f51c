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
    bad = [case.with_(nu=-0.1), case.with_(s_e=2.0), case.with_(varpi=1.0), case.with_(periodic_x=False)]
    fl = case.flags.copy(); fl[0, 0] = 7
    bad.append(case.with_(flags=fl))
    for b in bad:
        p, keep = P.make_params(b, "f32")
        assert L.lbm_footprint_bytes(C.byref(p)) == 0
        assert L.lbm_last_error(None)


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
