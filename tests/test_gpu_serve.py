"""Serving loop on the GPU: a request's result is the same (bit for bit) when
it is served alone and when it is served among others; the FP32-shifted
result of a served request is within 1e-4 (max-norm, relative to the field's
range) of the FP64 oracle after the same number of steps."""
import numpy as np
import pytest

import lbm_cases as lc
import oracle
from paper_1510_08224_gb300 import serve

pytestmark = pytest.mark.gpu


def _requests():
    stream = lc.serving_stream(n=6, seed=7, side_lo=16, side_hi=48)
    reqs = []
    for k, (t, kind, case) in enumerate(stream):
        sides = (0, 1) if kind == "cavity" else (2, 3)
        reqs.append(serve.Request(k, case, arrival=t, nusselt_sides=sides, want_fields=True))
    return reqs


def test_result_is_the_same_alone_and_in_the_mix():
    reqs = _requests()
    be = serve.GpuBackend("f32")
    srv = serve.Server(be, budget_bytes=150e9, check_every=250, tol=1e-6, step_cap=3000)
    mixed = {r.rid: r for r in srv.run(reqs, realtime=False)}
    assert srv.max_active == len(reqs)
    be.close()
    for req in reqs:
        be = serve.GpuBackend("f32")
        alone = serve.Server(be, check_every=250, tol=1e-6, step_cap=3000).run([req], realtime=False)[0]
        be.close()
        m = mixed[req.rid]
        assert alone.steps == m.steps and alone.nusselt == m.nusselt
        for a, b in zip(alone.fields, m.fields):
            assert np.array_equal(a, b)


def test_budget_admission_on_the_gpu():
    reqs = _requests()
    be = serve.GpuBackend("f32")
    fps = [be.footprint(r.case) for r in reqs]
    budget = max(fps) + min(fps)
    srv = serve.Server(be, budget_bytes=budget, check_every=250, tol=1e-6, step_cap=1000)
    res = srv.run(reqs, realtime=False)
    be.close()
    assert len(res) == len(reqs) and srv.peak_in_use <= budget


def test_served_fp32_result_against_the_fp64_oracle():
    case = lc.cavity(n=40, Ra=1e4, noise=1e-3)
    be = serve.GpuBackend("f32")
    res = serve.Server(be, check_every=500, tol=1e-6, step_cap=8000).run(
        [serve.Request(0, case, 0.0, nusselt_sides=(0,), want_fields=True)], realtime=False)[0]
    be.close()
    o = oracle.OracleLattice(case, threads=4)
    o.step(res.steps)
    _, ux, uy, T = res.fields
    _, uxo, uyo, To = o.macro()
    umax = max(np.abs(uxo).max(), np.abs(uyo).max())
    eu = max(np.abs(ux - uxo).max(), np.abs(uy - uyo).max()) / umax
    eT = np.abs(T - To).max() / case.delta_T
    print(f"served FP32 vs FP64 oracle after {res.steps} steps: u {eu:.2e}, T {eT:.2e}")
    assert eu <= 1e-4 and eT <= 1e-4
    assert abs(res.nusselt[0] - o.nusselt(0)) <= 1e-4 * o.nusselt(0)
