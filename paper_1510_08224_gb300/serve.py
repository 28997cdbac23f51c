"""Continuous-batching serving loop for lattice Boltzmann solves.

Requests (a problem each: cavity, Rayleigh-Benard, ...) arrive over time. A
request is admitted as soon as it has arrived and its device footprint
(lbm_footprint_bytes) fits in the remaining HBM budget; admitted lattices stay
resident and join the running batch, so new work overlaps on the device with
work already in flight. Every `check_every` steps each active lattice's
steady-state residual is read; a lattice that reaches `tol` or the step cap
leaves the batch, its result (Nusselt numbers, steps, residual, fields on
request) is recorded, and its memory returns to the budget.

Admission is first-come first-served in arrival order: a request that does not
fit blocks the ones behind it until memory frees up (no starvation of large
requests).

Every lattice is checked at the same step counts (multiples of `check_every`
after its admission) whether it runs alone or among others, and the batch
kernels give the same bits as a lattice stepped alone, so a request's result
does not depend on what else is being served.

The executor is pluggable: `GpuBackend` drives the CUDA library's batch
executor (every admitted request resident and stepped together; residuals of
all of them read with one synchronisation); `PlainBackend` is the plain path,
each request alone in FP64 storage with its own launches, run through the same
loop with one request admitted at a time (`max_active=1`), so its latencies
come from the same real-time stream. Tests of the scheduling logic use a fake
backend on the CPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time


@dataclasses.dataclass
class Request:
    rid: int
    case: object          # an lbm_cases.Case-like problem description
    arrival: float        # seconds after the start of the run
    nusselt_sides: tuple = ()   # wall sides whose mean Nusselt number to report
    want_fields: bool = False


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    residual: float
    converged: bool
    footprint: int
    cells: int
    nusselt: dict = dataclasses.field(default_factory=dict)
    fields: tuple | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class GpuBackend:
    """The CUDA library: lattices in torch device memory, one Batch of the
    given kind ('fused', 'persistent' or 'concurrent') and config (see
    Batch.set_config; -1 the default), optionally replayed from CUDA graphs of
    graph_steps steps."""

    def __init__(self, storage: str = "f32", graph_steps: int = 0, kind: str = "fused", steps_per_launch=None,
                 config: int = -1):
        import torch
        from . import lbm
        self._lbm = lbm
        self._torch = torch
        self.storage = storage
        self.batch = lbm.Batch()
        self.batch.set_kind(kind)
        if steps_per_launch is None:  # the persistent kind: one launch per replayed graph
            steps_per_launch = graph_steps if graph_steps > 0 else 32
        self.batch.set_mode(steps_per_launch, graph_steps)
        self.batch.set_config(config, 1)

    def footprint(self, case) -> int:
        p, keep = self._lbm.make_params(case, self.storage)
        return self._lbm.lbm_footprint_bytes(p)

    def create(self, case):
        return self._lbm.Lattice(case, storage=self.storage, stream=self.batch.stream)

    def add(self, lat):
        self.batch.add(lat)

    def remove(self, lat):
        self.batch.remove(lat)

    def step(self, n: int):
        self.batch.step(n)

    def residual(self, lat) -> float:
        return lat.residual()

    def residuals(self, lats) -> dict:
        """R of every resident lattice, one synchronisation (lbm_batch_residuals)."""
        r = self.batch.residuals()
        for lat in lats:
            if lat not in r:  # not batched (cannot happen in the server loop)
                r[lat] = lat.residual()
        return r

    def nusselt(self, lat, side) -> float:
        return lat.nusselt(side, 0.0, lat.case.delta_T)

    def fields(self, lat):
        return lat.macro()

    def release(self, lat):
        lat.close()

    def sync(self):
        self.batch.sync()

    def close(self):
        self.batch.close()


class PlainBackend:
    """The plain path: every lattice in FP64 storage stepped with its own
    launches (lbm_step), residuals read one lattice at a time."""

    def __init__(self, storage: str = "f64"):
        from . import lbm
        self._lbm = lbm
        self.storage = storage
        self.members = []

    def footprint(self, case) -> int:
        p, keep = self._lbm.make_params(case, self.storage)
        return self._lbm.lbm_footprint_bytes(p)

    def create(self, case):
        return self._lbm.Lattice(case, storage=self.storage)

    def add(self, lat):
        self.members.append(lat)

    def remove(self, lat):
        self.members.remove(lat)

    def step(self, n: int):
        for lat in self.members:
            lat.step(n)

    def residual(self, lat) -> float:
        return lat.residual()

    def nusselt(self, lat, side) -> float:
        return lat.nusselt(side, 0.0, lat.case.delta_T)

    def fields(self, lat):
        return lat.macro()

    def release(self, lat):
        lat.close()

    def sync(self):
        for lat in self.members:
            lat.sync()

    def close(self):
        self.members = []


class Server:
    def __init__(self, backend, budget_bytes: float = 150e9, check_every: int = 500, tol: float = 1e-6,
                 step_cap: int = 200_000, clock=time.perf_counter, sleep=time.sleep, max_active: int | None = None):
        self.backend = backend
        self.budget = float(budget_bytes)
        self.max_active_limit = max_active  # None: bounded by the budget alone
        self.check_every = int(check_every)
        self.tol = float(tol)
        # the cap is a whole number of checks, so every chunk is check_every steps
        self.step_cap = -(-int(step_cap) // self.check_every) * self.check_every
        self.clock = clock
        self.sleep = sleep
        self.in_use = 0
        self.peak_in_use = 0
        self.max_active = 0
        self.queued_for_memory = 0  # admissions that waited for memory to free up
        self.checks = 0             # residual checks (one per chunk)

    def _residuals(self, lats):
        f = getattr(self.backend, "residuals", None)
        if f is not None:
            return f(lats)
        return {lat: self.backend.residual(lat) for lat in lats}

    def run(self, requests, realtime: bool = True):
        """Serve `requests` (arrival times relative to the start). With
        realtime=False every request counts as arrived at time 0 (a closed
        batch). Returns the results in completion order."""
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        active = {}  # rid -> (request, lattice, steps, admitted, footprint)
        results = []
        waited = set()  # requests that found the budget full when they were next in line
        t0 = self.clock()

        def now():
            return self.clock() - t0

        while pending or active:
            t = now()
            # admission, first come first served
            while pending and (not realtime or pending[0].arrival <= t):
                if self.max_active_limit is not None and len(active) >= self.max_active_limit:
                    break
                req = pending[0]
                fp = self.backend.footprint(req.case)
                if fp > self.budget:
                    raise ValueError(f"request {req.rid} needs {fp} bytes, more than the whole budget")
                if self.in_use + fp > self.budget:
                    if req.rid not in waited:
                        self.queued_for_memory += 1
                        waited.add(req.rid)
                    break
                pending.popleft()
                lat = self.backend.create(req.case)
                self.backend.residual(lat)  # first call stores the snapshot
                self.backend.add(lat)
                self.in_use += fp
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                active[req.rid] = [req, lat, 0, now(), fp]
            self.max_active = max(self.max_active, len(active))
            if not active:
                if pending and realtime:
                    self.sleep(max(0.0, min(pending[0].arrival - now(), 0.01)))
                continue
            # one chunk of check_every steps for everything resident, then the checks
            self.backend.step(self.check_every)
            rs = self._residuals([a[1] for a in active.values()])
            self.checks += 1
            done = []
            for rid, a in active.items():
                a[2] += self.check_every
                r = rs[a[1]]
                if not r < self.tol and a[2] < self.step_cap and r == r:  # NaN: diverged, leaves at once
                    continue
                done.append((rid, r))
            for rid, r in done:
                req, lat, steps, admitted, fp = active.pop(rid)
                self.backend.remove(lat)
                nus = {s: self.backend.nusselt(lat, s) for s in req.nusselt_sides}
                fields = self.backend.fields(lat) if req.want_fields else None
                self.backend.release(lat)
                self.in_use -= fp
                cells = int((req.case.flags == 0).sum())
                results.append(Result(rid, req.arrival, admitted, now(), steps, r, r < self.tol, fp, cells, nus,
                                      fields))
        return results


def serial_baseline(backend_factory, requests, check_every: int, tol: float, step_cap: int,
                    clock=time.perf_counter):
    """The plain path: each request alone, one after another, with the same
    convergence checks. Returns (results, service times); latencies follow
    from a single-server queue over the arrival times."""
    step_cap = -(-int(step_cap) // check_every) * check_every
    service = {}
    results = []
    for req in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        be = backend_factory()
        t0 = clock()
        lat = be.create(req.case)
        be.residual(lat)
        steps = 0
        r = float("inf")
        while True:
            lat.step(check_every)
            steps += check_every
            r = be.residual(lat)
            if r < tol or steps >= step_cap:
                break
        nus = {s: be.nusselt(lat, s) for s in req.nusselt_sides}
        be.release(lat)
        service[req.rid] = clock() - t0
        results.append((req, steps, r, nus))
    # single-server FIFO queue over the measured service times
    t = 0.0
    out = []
    for req, steps, r, nus in results:
        start = max(t, req.arrival)
        t = start + service[req.rid]
        cells = int((req.case.flags == 0).sum())
        out.append(Result(req.rid, req.arrival, start, t, steps, r, r < tol, 0, cells, nus, None))
    return out, service


def percentile(values, q: float) -> float:
    """q-th percentile (0..100) by linear interpolation between order statistics."""
    v = sorted(values)
    if not v:
        return float("nan")
    k = (len(v) - 1) * q / 100.0
    lo = int(k)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


def summarize(results, makespan: float | None = None):
    lat = [r.latency for r in results]
    span = makespan if makespan is not None else (max(r.finished for r in results) if results else 0.0)
    return {
        "solves": len(results),
        "solves_per_s": len(results) / span if span > 0 else float("nan"),
        "p50_latency_s": percentile(lat, 50),
        "p99_latency_s": percentile(lat, 99),
        "converged": sum(r.converged for r in results),
        "cell_steps": sum(r.cells * r.steps for r in results),
    }


def summarize_converged(results):
    """Latency percentiles over the requests that reached steady state (their
    latency is the time to steady state), with their count and steps."""
    conv = [r for r in results if r.converged]
    lat = [r.latency for r in conv]
    steps = [r.steps for r in conv]
    return {"converged": len(conv), "of": len(results),
            "p50_time_to_steady_s": percentile(lat, 50), "p99_time_to_steady_s": percentile(lat, 99),
            "steps_p50": percentile(steps, 50), "steps_max": max(steps) if steps else None}
