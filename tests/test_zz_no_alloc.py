"""lbm_residual_fields_noalloc, the residual reduction for callers that cannot
call cudaMalloc (pre-budgeted serving loops, host frameworks that own the
allocator), checked through the C ABI against lbm_residual on the same
fields, on two calls in a row.

This file is collected last on purpose, so a run that stops at the first
failure has run every other test before it."""
import ctypes as C

import numpy as np
import pytest

import lbm_cases as lc

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_noalloc_residual_matches_lbm_residual_two_calls(storage):
    import torch
    import paper_1510_08224_gb300 as P
    L = P.load()
    case = lc.cavity(n=48, Ra=1e4, noise=1e-3)
    lat = P.Lattice(case, storage=storage)
    n = case.nx * case.ny
    solid = _dev((case.flags != 0).astype(np.uint8))
    stream = torch.cuda.current_stream()
    lat.step(20)
    assert np.isinf(lat.residual())  # first call: snapshot only
    prev = [_dev(a) for a in lat.macro()[1:]]
    for _ in range(2):
        lat.step(25)
        r_ref = lat.residual()
        cur = [_dev(a) for a in lat.macro()[1:]]
        r = C.c_double(-1.0)
        st = L.lbm_residual_fields_noalloc(cur[0].data_ptr(), cur[1].data_ptr(), cur[2].data_ptr(),
                                           prev[0].data_ptr(), prev[1].data_ptr(), prev[2].data_ptr(),
                                           solid.data_ptr(), C.c_int64(n), C.c_void_p(stream.cuda_stream),
                                           C.byref(r))
        assert st == 0, L.lbm_last_error(None)
        assert r_ref > 0 and abs(r.value - r_ref) <= 1e-12 * r_ref, (r.value, r_ref)
        prev = cur


def test_noalloc_residual_rejects_sizes_beyond_its_scratch():
    import paper_1510_08224_gb300 as P
    L = P.load()
    r = C.c_double()
    st = L.lbm_residual_fields_noalloc(None, None, None, None, None, None, None, C.c_int64(16_777_217), None,
                                       C.byref(r))
    assert st == 1 and b"16,777,216" in L.lbm_last_error(None)
