"""lbm_residual_fields_noalloc, the residual reduction for callers that cannot
call cudaMalloc (pre-budgeted serving loops, host frameworks that own the
allocator), checked through the C ABI against lbm_residual on the same
fields, and against the formula evaluated in NumPy (FP64), on two calls in a
row each time. The cases cover one reduction block, several blocks, a count
one cell past a whole number of blocks, the largest count the fixed scratch
takes, every cell counted (solid = NULL), the Python wrapper, and the refusal
of a capturing stream.

This file is collected last on purpose, so a run that stops at the first
failure has run every other test before it."""
import ctypes as C

import numpy as np
import pytest

import lbm_cases as lc

pytestmark = pytest.mark.gpu

MAX_CELLS = 16_777_216  # the entry point's documented limit (4096 blocks of 4096 cells)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()


def _call(L, cur, prev, solid, n, stream):
    r = C.c_double(-1.0)
    st = L.lbm_residual_fields_noalloc(cur[0].data_ptr(), cur[1].data_ptr(), cur[2].data_ptr(),
                                       prev[0].data_ptr(), prev[1].data_ptr(), prev[2].data_ptr(),
                                       None if solid is None else solid.data_ptr(), C.c_int64(n),
                                       C.c_void_p(stream.cuda_stream), C.byref(r))
    return st, r.value


def _numpy_residual(cur, prev, keep=None):
    """R = max(|u - u'|_2 / |u|_2, |T - T'|_2 / |T|_2), FP64, over the kept cells."""
    ux, uy, T = (np.asarray(a, np.float64) for a in cur)
    px, py, pT = (np.asarray(a, np.float64) for a in prev)
    if keep is not None:
        ux, uy, T, px, py, pT = (a[keep] for a in (ux, uy, T, px, py, pT))
    du = np.sqrt(np.sum((ux - px) ** 2 + (uy - py) ** 2)) / np.sqrt(np.sum(ux ** 2 + uy ** 2))
    dT = np.sqrt(np.sum((T - pT) ** 2)) / np.sqrt(np.sum(T ** 2))
    return max(du, dT)


@pytest.mark.parametrize("storage,case_name", [("f64", "cavity48"), ("f32", "cavity48"), ("f64", "rb256x128"),
                                               ("f32", "rb256x128")])
def test_noalloc_residual_matches_lbm_residual_two_calls(storage, case_name):
    """cavity 48 x 48 (2,500 cells: one block) and Rayleigh-Benard 256 x 128
    (33,280 cells: 9 blocks, the last one partial), fields read from a running
    lattice, against lbm_residual of the same lattice."""
    import torch
    import paper_1510_08224_gb300 as P
    L = P.load()
    if case_name == "cavity48":
        case = lc.cavity(n=48, Ra=1e4, noise=1e-3)
    else:
        case = lc.rayleigh_benard(nx=256, H=128, Ra=1e6, sigma=1e-2)
    lat = P.Lattice(case, storage=storage)
    n = case.nx * case.ny
    assert case_name == "cavity48" or n > 8 * 4096
    solid = _dev((case.flags != 0).astype(np.uint8))
    stream = torch.cuda.current_stream()
    lat.step(20)
    assert np.isinf(lat.residual())  # first call: snapshot only
    prev = [_dev(a) for a in lat.macro()[1:]]
    for _ in range(2):
        lat.step(25)
        r_ref = lat.residual()
        cur = [_dev(a) for a in lat.macro()[1:]]
        st, r = _call(L, cur, prev, solid, n, stream)
        assert st == 0, L.lbm_last_error(None)
        assert r_ref > 0 and abs(r - r_ref) <= 1e-12 * r_ref, (r, r_ref)
        prev = cur


@pytest.mark.parametrize("n", [3 * 4096 + 1, MAX_CELLS])
def test_noalloc_residual_every_cell_against_numpy(n):
    """solid = NULL (every cell counts) on seeded fields; a count one past three
    whole blocks, and exactly the largest count the scratch takes (4096
    blocks); two calls in a row with different fields."""
    import torch
    import paper_1510_08224_gb300 as P
    L = P.load()
    stream = torch.cuda.current_stream()
    for call in range(2):
        host = [lc.uniform01(100 + 10 * call + k, n) - 0.5 for k in range(6)]
        host[2] += 1.0  # T around 1
        host[5] += 1.0
        dev = [_dev(a) for a in host]
        st, r = _call(L, dev[:3], dev[3:], None, n, stream)
        assert st == 0, L.lbm_last_error(None)
        want = _numpy_residual(host[:3], host[3:])
        assert abs(r - want) <= 1e-12 * want, (call, r, want)
        del dev
    torch.cuda.empty_cache()


def test_noalloc_python_wrapper_with_and_without_solid():
    """residual_fields_noalloc on torch tensors equals Lattice.residual() with
    the solid mask, and the NumPy formula over every cell without it."""
    import torch
    import paper_1510_08224_gb300 as P
    case = lc.cavity(n=70, Ra=1e4, noise=1e-3)
    lat = P.Lattice(case, storage="f64")
    lat.step(10)
    lat.residual()
    prev = lat.macro()[1:]
    lat.step(30)
    r_ref = lat.residual()
    cur = lat.macro()[1:]
    solid = torch.from_numpy((case.flags != 0).astype(np.uint8).reshape(-1)).cuda()
    td = [_dev(a) for a in cur + prev]
    r = P.residual_fields_noalloc(*td, solid=solid)
    assert abs(r - r_ref) <= 1e-12 * r_ref, (r, r_ref)
    r_all = P.residual_fields_noalloc(*td)
    want = _numpy_residual([a.reshape(-1) for a in cur], [a.reshape(-1) for a in prev])
    assert abs(r_all - want) <= 1e-12 * want
    with pytest.raises(TypeError):
        P.residual_fields_noalloc(*[t.float() for t in td])
    with pytest.raises(ValueError):
        P.residual_fields_noalloc(td[0][:-1], *td[1:])


def test_noalloc_residual_refuses_a_capturing_stream():
    """The call copies its sums back and waits for its stream, which a stream
    capture forbids: on a capturing stream it returns LBM_EINVAL untouched."""
    import torch
    import paper_1510_08224_gb300 as P
    L = P.load()
    n = 5000
    dev = [_dev(lc.uniform01(7 + k, n) + 0.5) for k in range(6)]
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        st, _ = _call(L, dev[:3], dev[3:], None, n, s)
        g.capture_end()
    assert st == 1 and b"captured" in L.lbm_last_error(None)
    st, r = _call(L, dev[:3], dev[3:], None, n, torch.cuda.current_stream())
    assert st == 0 and np.isfinite(r)


def test_noalloc_residual_rejects_sizes_beyond_its_scratch():
    import paper_1510_08224_gb300 as P
    L = P.load()
    r = C.c_double()
    st = L.lbm_residual_fields_noalloc(None, None, None, None, None, None, None, C.c_int64(MAX_CELLS + 1), None,
                                       C.byref(r))
    assert st == 1 and b"16,777,216" in L.lbm_last_error(None)
