#!/usr/bin/env python3
"""Throughput of the fused non-orthogonal MRT D2Q9+D2Q5 step on one GB300.

Workload: Rayleigh-Benard cell, 4096 x 2048 fluid cells (plus the two wall
rows), periodic in x, Ra = 1e6, Pr = 0.71, Ma = 0.1, seeded 1e-3 Gaussian
temperature perturbation; FP32-shifted population storage by default.

One bench step = one time step of the whole lattice (one fused kernel launch).
value = fluid cells x steps / time / 1e6 (MLUPS), timed with CUDA events on the
lattice's stream, inputs resident in HBM. The working set (two population
buffers, > 1 GB) is far larger than L2, so no flush is needed between steps.

--impl reference times the FP64 CPU oracle on the host cores instead, each
step a bounded crop of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lbm_cases as lc  # noqa: E402

METRIC = "MLUPS (D2Q9+D2Q5) & % HBM roofline; solves/s and p50/p99 latency vs plain"
# algorithmic bytes per fluid-cell update: 14 populations read + written, plus the 1-byte link map
BYTES_PER_NODE = {"f64": 14 * 8 * 2 + 1, "f32": 14 * 4 * 2 + 1, "f16": 14 * 2 * 2 + 1}
STORAGE_NAME = {"f64": "f64", "f32": "f32-shifted", "f16": "f16-shifted"}
COMPUTE_DTYPE = {"f64": "f64", "f32": "f32", "f16": "f32"}
PROFILE_DIR = os.path.join(ROOT, "profiles")


def workload(nx: int, H: int):
    return lc.rayleigh_benard(nx=nx, H=H, Ra=1e6, Pr=0.71, Ma=0.1, seed=0, sigma=1e-3)


# The sources that define the single-lattice step kernels and how they are
# launched: the kernel translation units and every header they include (host
# code such as the batch executor or the C-ABI entry points is not part of it).
STEP_KERNEL_SOURCES = ("kernels_f64.cu", "kernels_f32.cu", "kernels_f16.cu", "launchers.cuh", "nomrt_kernels.cuh",
                       "nomrt_internal.h", "step8.cuh", "step_tma.cuh")


def kernel_source_hash() -> str:
    """Hash of the step kernels' sources: a committed ncu summary whose hash
    differs was taken on other kernels, and its counters are not reported."""
    d = os.path.join(ROOT, "paper_1510_08224_gb300", "csrc")
    h = hashlib.sha256()
    for name in STEP_KERNEL_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_values(name: str):
    """The key=value pairs of a committed ncu summary's header comment, or {}
    if the file is missing or the kernel sources changed since it was taken."""
    path = os.path.join(PROFILE_DIR, name)
    if not os.path.exists(path):
        return {}
    vals = {}
    with open(path) as f:
        for line in f:
            if line.startswith("<!--") and "=" in line:
                for kv in line.strip("<!- >\n").split():
                    if "=" in kv:
                        k, v = kv.split("=", 1)
                        vals[k] = v
    if vals.get("kernel_hash") != kernel_source_hash():
        return {}
    return vals


def profiled_traffic(storage: str, nx: int, ny: int):
    """DRAM bytes per step-kernel launch from the committed ncu summary, or None
    if there is none for this storage and size, or the kernel sources changed
    since it was taken."""
    try:
        return float(profile_values(f"k_step_{storage}_rb{nx}x{ny - 2}.md")["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# GB300's nominal FP64 rate (no measured FP64 peak exists for this machine); an FMA counts twice
FP64_PEAK_TFLOPS = 1.25


def fp64_alu_roofline(mlups: float):
    """The FP64 step kernel is bound by the FP64 pipe: achieved FP64 TFLOP/s from
    the ncu-counted DADD + DMUL + 2 DFMA per cell, against the nominal rate; also
    as FP64 instructions against half the nominal FLOP rate (the pipe's issue
    limit when every instruction counts once)."""
    v = profile_values("k_step_f64_rb1024x512.md")
    try:
        flops, inst = float(v["fp64_flops_per_cell"]), float(v["fp64_inst_per_cell"])
    except (KeyError, ValueError):
        return None
    tf = flops * mlups * 1e6 / 1e12
    ti = inst * mlups * 1e6 / 1e12
    return {"bound": "alu", "achieved": round(tf, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": round(tf / FP64_PEAK_TFLOPS, 4), "fp64_flops_per_cell": flops, "fp64_inst_per_cell": inst,
            "inst_frac": round(ti / (FP64_PEAK_TFLOPS / 2), 4),
            "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak); counts from ncu"}


class ClockSampler:
    """nvidia-smi samples (SM clock, max clock, throttle reasons) every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.samples = []
        self.proc = None
        self.gpu = gpu_index
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # the timed region is short: start it only once samples are flowing
        t_end = time.perf_counter() + 5.0
        while not self.samples and time.perf_counter() < t_end and self.proc.poll() is None:
            time.sleep(0.01)
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.perf_counter(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self, t0: float, t1: float):
        inside = [s for t, s in self.samples if t0 <= t <= t1]
        window = "timed"
        if not inside:
            inside = [s for _, s in self.samples]
            window = "run"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "window": "none"}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in inside:
            for k, n in enumerate(names):
                if s[4 + k].lower().startswith("active"):
                    reasons.add(n)

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(s[0]) for s in inside if num(s[0]) is not None]
        mx = [num(s[1]) for s in inside if num(s[1]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max_time(ms: float, dist, device) -> float:
    """Max over ranks of a per-rank time (the slowest rank bounds the job)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(fluid_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Cells all ranks updated (each rank advances its own replica) / slowest time."""
    return world * fluid_per_rank * steps / (ms_max * 1e-3) / 1e6


def time_steps(P, torch, case, storage, steps, warmup):
    """Device-timed K steps of one lattice. Returns (elapsed_ms, lattice)."""
    lat = P.Lattice(case, storage=storage)
    stream = torch.cuda.current_stream()
    lat.step(warmup)
    lat.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), lat


def e2e_run(P, torch, case, storage, steps):
    """End to end through the public API with host buffers: create from host
    flags and T_init (pinned), K steps, read rho, u, T back to host, destroy."""
    T_pinned = torch.empty(case.T_init.shape, dtype=torch.float64).pin_memory()
    T_pinned.numpy()[...] = case.T_init
    ecase = case.with_(T_init=T_pinned.numpy())
    out = [torch.empty((case.ny, case.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat = P.Lattice(ecase, storage=storage)
    lat.step(steps)
    import ctypes as C
    L = P.load()
    ptrs = [C.cast(o.data_ptr(), C.POINTER(C.c_double)) for o in out]
    st = L.lbm_read_macro(lat.handle, *ptrs)
    if st != 0:
        raise RuntimeError(L.lbm_last_error(lat.handle).decode())
    lat.close()
    t1 = time.perf_counter()
    h2d = case.nx * case.ny * (8 + 1)  # T_init + flags
    d2h = 4 * 8 * case.nx * case.ny
    return (t1 - t0), h2d, d2h


def _oracle_mlups(case, threads: int, target_s: float):
    """The oracle as it stands on `threads` host cores: steps timed for ~target_s."""
    import oracle
    o = oracle.OracleLattice(case, threads=threads)
    o.step(1)
    t0 = time.perf_counter()
    o.step(2)
    per = (time.perf_counter() - t0) / 2
    n = max(3, int(target_s / max(per, 1e-6)))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    return case.fluid_nodes * n / dt / 1e6, n, dt


def cpu_baseline(case_full, target_s: float = 12.0, crop=(512, 256)):
    """The FP64 oracle as it stands on the host cores, on a crop of the
    workload (same nu, alpha, g beta; crop x crop cells), timed for ~target_s
    on all cores; also on one core, and the 256 x 256 cavity at Ra = 1e5 on
    all cores and on one core (a few seconds each)."""
    import oracle
    threads = min(os.cpu_count() or 1, oracle.threads_available())
    cx, cy = crop
    crop_case = lc.rayleigh_benard(nx=cx, H=cy, Ra=1e6, Pr=0.71, Ma=0.1, seed=0, sigma=1e-3, L=case_full.L)
    mlups, n, dt = _oracle_mlups(crop_case, threads, target_s)
    m1, n1, dt1 = _oracle_mlups(crop_case, 1, target_s / 3)
    cav = lc.cavity(n=256, Ra=1e5, Pr=0.71, Ma=0.1, seed=0, noise=1e-6)
    mc, nc, dtc = _oracle_mlups(cav, threads, target_s / 3)
    mc1, nc1, dtc1 = _oracle_mlups(cav, 1, target_s / 4)
    return {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"{cx}x{cy} crop of the workload (same nu, alpha, g beta), {n} steps, {dt:.1f} s, "
                      f"FP64 C oracle, OpenMP over rows",
            "single_thread": {"value": round(m1, 3), "unit": "MLUPS", "cores": 1,
                              "sample": f"same crop, {n1} steps, {dt1:.1f} s"},
            "cavity_256_ra1e5": {"value": round(mc, 3), "unit": "MLUPS", "cores": threads,
                                 "sample": f"256x256 cavity, {nc} steps, {dtc:.1f} s",
                                 "single_thread": {"value": round(mc1, 3), "unit": "MLUPS", "cores": 1,
                                                   "sample": f"same cavity, {nc1} steps, {dtc1:.1f} s"}}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    nx, H = args.nx, args.H
    case_full = workload(nx, H)
    threads = min(os.cpu_count() or 1, oracle.threads_available())
    cx, cy = min(nx, 256), min(H, 128)
    crop_case = lc.rayleigh_benard(nx=cx, H=cy, Ra=1e6, Pr=0.71, Ma=0.1, seed=0, sigma=1e-3, L=case_full.L)
    o = oracle.OracleLattice(crop_case, threads=threads)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = crop_case.fluid_nodes * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"rayleigh_benard_{nx}x{H}_ra1e6", "nx": nx, "ny": H, "storage": "f64 (CPU oracle)",
                   "sample": f"each step: one {cx}x{cy} crop step"},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": f"{cx}x{cy} crop of the workload, {args.steps} steps"},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    """Batched uneven lattices: 64 differentially heated cavities, sides drawn
    over 128..1024, Ra log-uniform in [1e3, 1e6], advanced together; compared
    with stepping each lattice with its own launches."""
    import torch
    import paper_1510_08224_gb300 as P
    torch.cuda.set_device(0)
    cases = lc.batched_cavities(count=args.count, seed=0)
    cells = sum(c.fluid_nodes for c in cases)
    lats = [P.Lattice(c, storage=args.storage) for c in cases]
    stream = torch.cuda.current_stream()
    b = P.Batch()
    for lat in lats:
        b.add(lat)
    best, best_rows, ms_cfg = b.tune(trial_launches=5)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, steps):
        fn(args.warmup)
        torch.cuda.synchronize()
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    res = {}
    tuned_kind = b.info()["config"]
    for name, mode, kind in (("fused_graph", (1, 32), "fused"), ("fused_launch_per_step", (1, 0), "fused"),
                             ("fused_persistent_8", (8, 0), "fused"), ("concurrent_graph", (1, 32), "concurrent"),
                             ("concurrent_graph_2", (1, 2), "concurrent")):
        b.set_kind(kind)
        b.set_mode(*mode)
        ms = timed(b.step, args.steps)
        res[name] = {"MLUPS": round(cells * args.steps / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms / args.steps, 4)}
    b.close()

    def serial(n):
        for _ in range(n):
            for lat in lats:
                lat.step(1)
    ms_serial = timed(serial, max(10, args.steps // 10))
    k_serial = max(10, args.steps // 10)
    best_mode = min(res, key=lambda k: res[k]["ms_per_step"])
    best_ms = res[best_mode]["ms_per_step"]
    best_kernel = ("k_step4 of every member, concurrent streams" if best_mode.startswith("concurrent")
                   else "k_batch_persistent" if "persistent" in best_mode else "k_batch_grid")
    value = cells / (best_ms * 1e-3) / 1e6
    peak, peak_src = measured_peak()
    achieved = BYTES_PER_NODE[args.storage] * cells / (best_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(best_ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": COMPUTE_DTYPE[args.storage], "data": "synthetic",
        "config": {"workload": f"batched_cavities_{args.count}", "lattices": args.count, "fluid_cells": cells,
                   "sides": "uniform 128..1024", "Ra": "log-uniform [1e3, 1e6]", "storage": STORAGE_NAME[args.storage],
                   "tuned_config": best, "tuned_rows_per_unit": best_rows,
                   "tune_ms_per_launch": {k: round(m, 4) for k, m in ms_cfg.items()}},
        "modes": res,
        "serial_per_lattice": {"MLUPS": round(cells * k_serial / (ms_serial * 1e-3) / 1e6, 1),
                               "ms_per_step": round(ms_serial / k_serial, 4), "launches_per_step": args.count},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None, "kernel": best_kernel, "mode": best_mode,
                     "peak_source": f"{peak_src} HBM copy bandwidth (burst)"},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_cost(args):
    """Cost of the collision operators and temperature lattices on the same
    workload (Rayleigh-Benard, --nx x --H): MRT (Eq. 8 + Eq. 24) against BGK,
    with D2Q5 (Sec. 2.2) or the D2Q9 temperature model (Eqs. 31-33), in each
    storage. Per model: the AUTO kernel and every step kernel of the storage
    (scalar, VEC4 configs), device-timed; the line's value is the MRT D2Q5
    MLUPS of --storage."""
    import torch
    import paper_1510_08224_gb300 as P
    torch.cuda.set_device(0)
    base = workload(args.nx, args.H)
    fluid = base.fluid_nodes
    peak, peak_src = measured_peak()
    models = {"mrt_d2q5": base, "bgk_d2q5": lc.with_bgk(base),
              "mrt_d2q9t": lc.with_d2q9_temperature(base), "bgk_d2q9t": lc.with_bgk(lc.with_d2q9_temperature(base))}
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(0).start()
    t_start = time.perf_counter()
    table = {}
    launches = 0
    for st in ("f64", "f32", "f16"):
        eb = {"f64": 8, "f32": 4, "f16": 2}[st]
        k = args.steps if st != "f64" else max(10, args.steps // 8)
        for name, case in models.items():
            planes = 9 + (9 if case.thermal_q == 9 else 5)
            bpn = planes * eb * 2 + 1
            lat = P.Lattice(case, storage=st)
            kernels = [("auto", 0)]
            if st != "f64" and args.sweep:
                kernels += [("scalar", 0)] + [("vec4", c) for c in range(P.step_kernel_count(st, "vec4"))]
            row = {}
            for v in kernels:
                lat.set_step_kernel(*v)
                lat.step(args.warmup)
                lat.sync()
                e0.record(stream)
                lat.step(k)
                e1.record(stream)
                e1.synchronize()
                launches += k
                ms = e0.elapsed_time(e1) / k
                gbs = bpn * fluid / (ms * 1e-3) / 1e9
                row[f"{v[0]}{v[1] if v[0] == 'vec4' else ''}"] = {
                    "MLUPS": round(fluid / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms, 5),
                    "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4)}
            try:  # the timing does not depend on it, but say whether the run stayed finite
                lat.residual()
                finite = True
            except P.LBMError:
                finite = False
            lat.close()
            table[f"{st}/{name}"] = {"bytes_per_node": bpn, "steps": k, "finite": finite, "kernels": row}
    t_end = time.perf_counter()
    sampler.stop()

    def best_ms(key):
        return min(v["ms_per_step"] for v in table[key]["kernels"].values())

    ratios = {}
    for st in ("f64", "f32", "f16"):
        m5, b5 = best_ms(f"{st}/mrt_d2q5"), best_ms(f"{st}/bgk_d2q5")
        m9, b9 = best_ms(f"{st}/mrt_d2q9t"), best_ms(f"{st}/bgk_d2q9t")
        ratios[st] = {"mrt_over_bgk_d2q5": round(m5 / b5, 4), "mrt_over_bgk_d2q9t": round(m9 / b9, 4),
                      "d2q9t_over_d2q5_mrt": round(m9 / m5, 4)}
    key = f"{args.storage}/mrt_d2q5"
    ms = table[key]["kernels"]["auto"]["ms_per_step"]
    line = {
        "metric": METRIC, "value": round(fluid / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": COMPUTE_DTYPE[args.storage], "data": "synthetic",
        "config": {"workload": f"collision_cost_rayleigh_benard_{args.nx}x{args.H}", "fluid_cells": fluid,
                   "storage": STORAGE_NAME[args.storage],
                   "models": "MRT or BGK collisions; D2Q5 or D2Q9 temperature lattice",
                   "l2": "no flush: working set > L2"},
        "models": table,
        "time_ratios_best_kernel": ratios,
        "gpu_launches": launches,
        "clocks": sampler.summary(t_start, t_end),
        "peak": {"hbm_gbs": peak, "source": peak_src},
    }
    print(json.dumps(line), flush=True)
    return 0


def cavity_table3_quantities(case, rho, ux, uy, T):
    """The quantities of Table 3 (Sec. 3.4) from the steady fields of a
    node-based cavity (walls on the boundary nodes, n intervals, L = n):
    u_x max on the vertical midline and u_y max on the horizontal midline in
    units of alpha / L, with their positions; the local Nusselt number on the
    cold wall, -L (dT/dx)_wall / dT with the second-order one-sided gradient
    (3 T_w - 4 T_1 + T_2) / 2 taken toward the wall, its maximum and position,
    and its mean by the trapezoidal rule over the wall."""
    n = case.nx - 1
    scale = n / case.alpha
    mid = n // 2
    col = ux[:, mid] * scale
    row = uy[mid, :] * scale
    jy, ix = int(np.argmax(col)), int(np.argmax(row))
    Tw = T[:, n]
    grad = (3.0 * Tw - 4.0 * T[:, n - 1] + T[:, n - 2]) / 2.0   # dT/dx at x = L
    nu_loc = -n * grad / case.delta_T
    jn = int(np.argmax(nu_loc))
    nu_mean = float(np.sum((nu_loc[1:] + nu_loc[:-1]) / 2.0) / n)
    # the volume form, a diagnostic: Nu = 1 + L <u_x T> / (alpha dT), trapezoidal average
    # over the node grid (conduction carries alpha dT / L on average, advection the rest)
    wts = np.ones(n + 1)
    wts[0] = wts[-1] = 0.5
    avg = float(wts @ (ux * T) @ wts) / (n * n)
    nu_vol = 1.0 + n * avg / (case.alpha * case.delta_T)
    return {"ux_max": float(col[jy]), "y_max": jy / n, "uy_max": float(row[ix]), "x_max": ix / n,
            "Nu_max": float(nu_loc[jn]), "y_Nu": jn / n, "Nu_mean": nu_mean, "Nu_vol": nu_vol}


def run_table3(args):
    """Table 3 of the paper (natural convection in a square cavity, Pr = 0.71,
    Ma = 0.1, the paper's node-based walls and grids), each Ra run to a
    steady-state residual below 1e-10, FP64 storage."""
    import torch
    import paper_1510_08224_gb300 as P
    torch.cuda.set_device(0)
    table = np.loadtxt(os.path.join(ROOT, "tests", "golden", "table3_cavity.txt"))
    rows = {}
    t0 = time.perf_counter()
    for Ra, grid, uxp, uyp, nmaxp, nmeanp in table:
        case = lc.cavity_nee(n=int(grid), Ra=float(Ra))
        lat = P.Lattice(case, storage=args.storage)
        lat.residual()
        steps, r = 0, float("inf")
        while r >= 1e-10 and steps < 3_000_000:
            lat.step(2000)
            steps += 2000
            r = lat.residual()
        q = cavity_table3_quantities(case, *lat.macro())
        q["Nu_mean_hot_library"] = lat.nusselt("left", L=float(grid))
        q.update(steps=steps, residual=r)
        q["paper"] = {"ux_max": uxp, "uy_max": uyp, "Nu_max": nmaxp, "Nu_mean": nmeanp}
        q["rel_dev"] = {k: round((q[k] - v) / v, 5) for k, v in q["paper"].items()}
        rows[f"{Ra:g}"] = q
        lat.close()
    line = {"metric": METRIC, "value": max(abs(v) for q in rows.values() for v in q["rel_dev"].values()),
            "unit": "max relative deviation from Table 3", "n_gpus": 1, "higher_is_better": False,
            "dtype": COMPUTE_DTYPE[args.storage], "data": "synthetic",
            "config": {"workload": "table3_cavity_nee", "storage": STORAGE_NAME[args.storage],
                       "walls": "node-based, non-equilibrium extrapolation", "Pr": 0.71, "Ma": 0.1,
                       "steady": "residual < 1e-10, checked every 2000 steps"},
            "rows": rows, "seconds": round(time.perf_counter() - t0, 1)}
    print(json.dumps(line), flush=True)
    return 0


def serving_measure(storage: str, count: int, side_hi: int, step_cap: int, check_every: int, graph_steps: int):
    """Continuous-batching serving: Poisson arrivals (20 per second, seed 0) of
    `count` cavity and Rayleigh-Benard requests, sides log-uniform in
    [64, side_hi], Ra log-uniform in [1e3, 1e6], each run to residual < 1e-6 or
    the step cap, admitted by a 150 GB HBM budget; against the plain path (FP64
    storage, one request at a time, same convergence checks). Returns (config,
    served, plain) dictionaries."""
    import torch
    from paper_1510_08224_gb300 import serve
    torch.cuda.set_device(0)
    stream = lc.serving_stream(n=count, seed=0, side_lo=64, side_hi=side_hi)
    reqs = [serve.Request(k, c, t, nusselt_sides=((0,) if kind == "cavity" else (2,))) for k, (t, kind, c) in
            enumerate(stream)]
    cells = sum(int((r.case.flags == 0).sum()) for r in reqs)
    be = serve.GpuBackend(storage, graph_steps=graph_steps)
    srv = serve.Server(be, budget_bytes=150e9, check_every=check_every, tol=1e-6, step_cap=step_cap)
    t0 = time.perf_counter()
    res = srv.run(reqs, realtime=True)
    span = time.perf_counter() - t0
    be.close()
    s_ours = serve.summarize(res, span)
    base, service = serve.serial_baseline(lambda: serve.GpuBackend("f64"), reqs, check_every, 1e-6, step_cap)
    s_base = serve.summarize(base)
    same_steps = sum(1 for a, b in zip(sorted(res, key=lambda r: r.rid), sorted(base, key=lambda r: r.rid))
                     if a.steps == b.steps)
    config = {"workload": f"serving_stream_{count}", "arrivals": "Poisson 20/s, seed 0",
              "sides": f"log-uniform [64, {side_hi}]", "Ra": "log-uniform [1e3, 1e6]",
              "types": "cavity | rayleigh_benard", "tol": 1e-6, "step_cap": srv.step_cap,
              "check_every": check_every, "hbm_budget_bytes": 150e9, "storage": STORAGE_NAME[storage],
              "requests": len(reqs), "fluid_cells_total": cells, "graph_steps": graph_steps}
    served = {**s_ours, "makespan_s": round(span, 3), "peak_hbm_bytes": srv.peak_in_use,
              "max_concurrent": srv.max_active, "MLUPS": round(s_ours["cell_steps"] / span / 1e6, 1)}
    plain = {**s_base, "service_s_total": round(sum(service.values()), 3),
             "MLUPS": round(s_base["cell_steps"] / sum(service.values()) / 1e6, 1), "same_step_counts": same_steps}
    return config, served, plain


def run_serving(args):
    """The serving stream as its own bench line (value = solves/s)."""
    config, served, plain = serving_measure(args.storage, args.count, args.side_hi, args.step_cap,
                                            args.check_every, args.graph_steps)
    line = {
        "metric": METRIC, "value": round(served["solves_per_s"], 4), "unit": "solves/s", "n_gpus": 1,
        "steps": config["step_cap"], "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": COMPUTE_DTYPE[args.storage], "data": "synthetic", "config": config,
        "served": served, "plain_fp64_serial": plain,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "f64"])
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--H", type=int, default=2048)
    ap.add_argument("--variant", default="auto", choices=["auto", "scalar", "vec4", "vec8", "tma"],
                    help="step kernel variant (lbm_set_step_kernel)")
    ap.add_argument("--config", type=int, default=0, help="shape index of the step variant")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="rb: skip the short serving stream")
    ap.add_argument("--sweep", action="store_true", help="cost workload: time every step kernel of each model")
    ap.add_argument("--workload", default="rb", choices=["rb", "batch", "serve", "cost", "table3"],
                    help="rb: the 4096 x 2048 Rayleigh-Benard step (default); batch: uneven cavities advanced together; serve: the serving stream; cost: collision operators; table3: the cavity of Table 3")
    ap.add_argument("--count", type=int, default=64, help="lattices (batch) or requests (serve)")
    ap.add_argument("--side-hi", type=int, default=2048, help="largest side of a served request")
    ap.add_argument("--step-cap", type=int, default=20000, help="step cap of a served request")
    ap.add_argument("--check-every", type=int, default=500, help="steps between residual checks (serve)")
    ap.add_argument("--graph-steps", type=int, default=20,
                    help="serve: steps per captured CUDA graph of the served batch (0: launches from the host)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batched(args)
    if args.workload == "serve":
        return run_serving(args)
    if args.workload == "cost":
        return run_cost(args)
    if args.workload == "table3":
        return run_table3(args)

    import torch
    import paper_1510_08224_gb300 as P

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    case = workload(args.nx, args.H)
    fluid = case.fluid_nodes
    sampler = ClockSampler(local).start()
    # every rank advances its own replica of the workload (independent lattices)
    lat = P.Lattice(case, storage=args.storage)
    lat.set_step_kernel(args.variant, args.config)
    stream = torch.cuda.current_stream()
    lat.step(args.warmup)
    lat.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = time.perf_counter()
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    t_end = time.perf_counter()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    ms_max = reduce_max_time(ms, dist, "cuda")
    sampler.stop()
    clocks = sampler.summary(t_start, t_end)
    r = lat.residual()  # finite-state check of the run (first call: snapshot)
    lat.close()
    del lat

    value = whole_job_mlups(fluid, args.steps, world, ms_max)
    ms_step = ms_max / args.steps
    peak, peak_src = measured_peak()
    achieved = BYTES_PER_NODE[args.storage] * fluid / (ms / args.steps * 1e-3) / 1e9
    traffic = profiled_traffic(args.storage, args.nx, args.H + 2)
    roof = {"bound": "hbm" if args.storage != "f64" else "alu", "achieved": round(achieved, 1),
            "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "kernel": "k_step", "bytes_per_node": BYTES_PER_NODE[args.storage],
            "peak_source": f"{peak_src} HBM copy bandwidth (burst)"}
    if args.storage == "f64":
        alu = fp64_alu_roofline(value / world)
        if alu:
            alu["hbm_GB/s"] = roof["achieved"]
            alu["hbm_frac"] = roof["frac"]
            roof = alu

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": COMPUTE_DTYPE[args.storage], "data": "synthetic",
        "config": {"workload": f"rayleigh_benard_{args.nx}x{args.H}_ra1e6", "nx": args.nx, "ny": args.H,
                   "fluid_cells": fluid, "storage": STORAGE_NAME[args.storage],
                   "l2": "no flush: working set > L2 (two population buffers of "
                         f"{BYTES_PER_NODE[args.storage] // 2 * fluid / 1e9:.2f} GB each)",
                   "parallelism": f"replicas{world}", "step_kernel": [args.variant, args.config]},
        "roofline": roof,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "residual_check": r,
    }

    if rank == 0 and not args.no_e2e:
        e2e_steps = args.steps
        secs, h2d, d2h = e2e_run(P, torch, case, args.storage, e2e_steps)
        line["e2e"] = {"value": round(fluid * e2e_steps / secs / 1e6, 1), "unit": "MLUPS",
                       "h2d_bytes_per_step": int(h2d / e2e_steps), "d2h_bytes_per_step": int(d2h / e2e_steps),
                       "what": "lbm_create from pinned host flags+T_init, lbm_step(K), lbm_read_macro to pinned "
                               "host, lbm_destroy; wall clock"}
    if rank == 0 and not args.no_variants:
        var = {}
        for st in ("f32", "f16", "f64"):
            if st == args.storage:
                continue
            k = max(10, min(args.steps, 500))
            vms, vl = time_steps(P, torch, case, st, k, args.warmup)
            vl.close()
            vach = BYTES_PER_NODE[st] * fluid / (vms / k * 1e-3) / 1e9
            vm = fluid * k / (vms * 1e-3) / 1e6
            var[STORAGE_NAME[st]] = {"MLUPS": round(vm, 1), "steps": k,
                                     "GB/s": round(vach, 1), "frac": round(vach / peak, 4)}
            if st == "f64":
                var[STORAGE_NAME[st]]["alu"] = fp64_alu_roofline(vm)
        line["variants"] = var
    if rank == 0 and world == 1 and not args.no_serving:
        # the metric's second half (solves/s, p50/p99 latency against the plain path) on
        # a shorter stream than --workload serve, so that the default run stays short
        try:
            config, served, plain = serving_measure(args.storage if args.storage != "f64" else "f32", 16, 1024,
                                                    10000, 500, args.graph_steps)
            line["serving"] = {"config": config, "served": served, "plain_fp64_serial": plain,
                               "speedup_solves_per_s": round(served["solves_per_s"] / plain["solves_per_s"], 2),
                               "p99_latency_ratio": round(plain["p99_latency_s"] / served["p99_latency_s"], 2)}
        except Exception as exc:  # the step measurement above stands on its own
            line["serving"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(case)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
