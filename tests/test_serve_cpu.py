"""Scheduling logic of the serving loop on the CPU, with a fake executor:
admission by footprint within the budget, first-come first-served order,
overlap of requests, and results independent of the mix."""
import numpy as np

import lbm_cases as lc
from paper_1510_08224_gb300 import serve


class FakeLattice:
    def __init__(self, case):
        self.case = case
        self.steps = 0
        self.rate = 1.0 / (1 + case.meta.get("k", 0) % 3)  # convergence speed differs per request

    def step(self, n):
        self.steps += n

    def residual(self):
        return 10.0 ** (-self.rate * self.steps / 500.0)


class FakeBackend:
    def __init__(self):
        self.members = set()
        self.created = 0

    def footprint(self, case):
        return int(case.nx * case.ny * 100)

    def create(self, case):
        self.created += 1
        return FakeLattice(case)

    def add(self, lat):
        self.members.add(lat)

    def remove(self, lat):
        self.members.remove(lat)

    def step(self, n):
        for m in self.members:
            m.step(n)

    def residual(self, lat):
        return lat.residual()

    def nusselt(self, lat, side):
        return 1.0 + lat.steps

    def fields(self, lat):
        return None

    def release(self, lat):
        pass


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t

    def sleep(self, dt):
        self.t += dt


def _requests(n=12):
    reqs = []
    for k in range(n):
        c = lc.couette(H=8 + 4 * (k % 4), nx=4 + k)
        c.meta["k"] = k
        reqs.append(serve.Request(k, c, arrival=0.01 * k, nusselt_sides=(2,)))
    return reqs


def test_budget_is_never_exceeded_and_all_requests_finish():
    reqs = _requests()
    fps = [FakeBackend().footprint(r.case) for r in reqs]
    budget = 2.5 * max(fps)
    clock = FakeClock()
    srv = serve.Server(FakeBackend(), budget_bytes=budget, check_every=100, tol=1e-4, step_cap=10_000, clock=clock,
                       sleep=clock.sleep)
    res = srv.run(reqs)
    assert sorted(r.rid for r in res) == list(range(len(reqs)))
    assert srv.peak_in_use <= budget
    assert srv.max_active >= 2  # requests overlap
    for r in res:
        assert r.admitted >= r.arrival and r.finished >= r.admitted
        assert r.steps % 100 == 0 and r.converged


def test_first_come_first_served_admission():
    reqs = _requests(6)
    budget = max(FakeBackend().footprint(r.case) for r in reqs)  # one at a time
    clock = FakeClock()
    srv = serve.Server(FakeBackend(), budget_bytes=budget, check_every=100, tol=1e-4, clock=clock, sleep=clock.sleep)
    res = srv.run(reqs)
    order = sorted(res, key=lambda r: r.admitted)
    assert [r.rid for r in order] == sorted(r.rid for r in res)


def test_result_does_not_depend_on_the_mix():
    reqs = _requests(8)
    clock = FakeClock()
    mixed = {r.rid: r for r in serve.Server(FakeBackend(), check_every=100, tol=1e-4, clock=clock,
                                            sleep=clock.sleep).run(reqs)}
    for req in reqs:
        alone = serve.Server(FakeBackend(), check_every=100, tol=1e-4, clock=clock, sleep=clock.sleep).run([req])[0]
        assert alone.steps == mixed[req.rid].steps and alone.nusselt == mixed[req.rid].nusselt


def test_percentiles_and_summary():
    assert serve.percentile([1, 2, 3, 4], 50) == 2.5
    assert serve.percentile([5], 99) == 5
    rs = [serve.Result(k, 0.0, 0.0, float(k + 1), 100, 1e-7, True, 0, 10) for k in range(4)]
    s = serve.summarize(rs)
    assert s["solves"] == 4 and abs(s["solves_per_s"] - 1.0) < 1e-12 and s["p50_latency_s"] == 2.5


def test_serial_baseline_queue():
    reqs = _requests(4)
    clock = FakeClock()
    res, service = serve.serial_baseline(FakeBackend, reqs, check_every=100, tol=1e-4, step_cap=10_000, clock=clock)
    t = 0.0
    for r in res:
        start = max(t, r.arrival)
        assert abs(r.admitted - start) < 1e-12
        t = r.finished


def test_serving_stream_is_seeded():
    a = lc.serving_stream(n=10, seed=3, side_hi=256)
    b = lc.serving_stream(n=10, seed=3, side_hi=256)
    assert [x[0] for x in a] == [x[0] for x in b]
    assert all(np.array_equal(x[2].flags, y[2].flags) for x, y in zip(a, b))
    gaps = np.diff([x[0] for x in lc.serving_stream(n=400, seed=1, side_hi=64)])
    assert abs(gaps.mean() - 1 / 20.0) < 0.25 / 20.0  # Poisson arrivals at 20 per second


class FakeBatchBackend(FakeBackend):
    """Reads every resident lattice's residual in one call, as GpuBackend does."""

    def __init__(self):
        super().__init__()
        self.calls = 0

    def residuals(self, lats):
        self.calls += 1
        return {lat: lat.residual() for lat in lats}


def test_batched_residual_checks_and_queueing_for_memory():
    """One residual call per chunk for all resident lattices; a budget of two
    requests makes the rest wait for memory, and the count says so."""
    reqs = _requests(8)
    fps = [FakeBackend().footprint(r.case) for r in reqs]
    budget = sorted(fps)[-1] + sorted(fps)[-2]
    clock = FakeClock()
    be = FakeBatchBackend()
    srv = serve.Server(be, budget_bytes=budget, check_every=100, tol=1e-4, clock=clock, sleep=clock.sleep)
    res = srv.run(reqs, realtime=False)
    assert len(res) == 8 and be.calls == srv.checks
    assert srv.queued_for_memory >= 1 and srv.peak_in_use <= budget


def test_max_active_one_serves_one_request_at_a_time():
    """The plain path's admission: one request at a time, in arrival order,
    each admitted when the previous one leaves."""
    reqs = _requests(5)
    clock = FakeClock()
    srv = serve.Server(FakeBackend(), check_every=100, tol=1e-4, clock=clock, sleep=clock.sleep, max_active=1)
    res = srv.run(reqs)
    assert srv.max_active == 1
    order = sorted(res, key=lambda r: r.admitted)
    assert [r.rid for r in order] == [r.rid for r in sorted(reqs, key=lambda q: q.arrival)]
    for a, b in zip(order, order[1:]):
        assert b.admitted >= a.finished


def test_summary_over_converged_requests():
    rs = [serve.Result(k, 0.0, 0.0, float(k + 1), 100 * (k + 1), 1e-7 if k < 3 else 1e-3, k < 3, 0, 10)
          for k in range(4)]
    s = serve.summarize_converged(rs)
    assert s["converged"] == 3 and s["of"] == 4
    assert s["p50_time_to_steady_s"] == 2.0 and s["steps_max"] == 300
