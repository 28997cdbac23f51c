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


# GB300's nominal FP64 rate, for context beside the measured one; an FMA counts twice
FP64_NOMINAL_TFLOPS = 1.25


def fp64_alu_roofline(mlups: float, dfma_per_s: float | None):
    """The FP64 step kernel is bound by the FP64 pipe: its ncu-counted FP64
    instructions per cell (DADD + DMUL + DFMA) times the cell rate, against
    the DFMA instruction rate measured on this device by lbm_probe_fp64_rate
    (one instruction per clock and pipe lane, like DADD and DMUL); also as
    TFLOP/s (DFMA counting twice) against twice that rate."""
    v = profile_values("k_step_f64_rb1024x512.md")
    try:
        flops, inst = float(v["fp64_flops_per_cell"]), float(v["fp64_inst_per_cell"])
    except (KeyError, ValueError):
        return None
    ti = inst * mlups * 1e6
    tf = flops * mlups * 1e6 / 1e12
    out = {"bound": "alu", "fp64_flops_per_cell": flops, "fp64_inst_per_cell": inst,
           "achieved_tflops": round(tf, 4), "nominal_tflops": FP64_NOMINAL_TFLOPS}
    if dfma_per_s:
        out.update({"achieved": round(ti / 1e12, 4), "peak": round(dfma_per_s / 1e12, 4), "unit": "Tinst/s",
                    "frac": round(ti / dfma_per_s, 4), "peak_tflops": round(2 * dfma_per_s / 1e12, 4),
                    "flop_frac": round(tf / (2 * dfma_per_s / 1e12), 4),
                    "peak_source": "measured: lbm_probe_fp64_rate (independent DFMA chains, best of 5)"})
    else:
        out.update({"achieved": round(tf, 4), "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                    "frac": round(tf / FP64_NOMINAL_TFLOPS, 4), "peak_source": "nominal (no measurement)"})
    return out


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


def host_link_gbs(torch, nbytes: int = 256 << 20, reps: int = 5):
    """Pinned host <-> device copy rates (best of reps, CUDA events), GB/s."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = {}
    for name, dst, src in (("h2d", d, h), ("d2h", h, d)):
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            dst.copy_(src, non_blocking=True)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = round(nbytes / (best * 1e-3) / 1e9, 1)
    del h, d
    return out


def e2e_run(P, torch, case, storage, steps):
    """End to end through the public API with host buffers: footprint query,
    lbm_create from pinned host flags and T_init (device block from torch), K
    steps, read rho, u, T back to pinned host, destroy; wall clock, with the
    time of each phase (a stream synchronisation after the steps separates the
    steps from the read-back; lbm_read_macro waits for them anyway)."""
    import ctypes as C
    L = P.load()
    T_pinned = torch.empty(case.T_init.shape, dtype=torch.float64).pin_memory()
    T_pinned.numpy()[...] = case.T_init
    F_pinned = torch.empty(case.flags.shape, dtype=torch.uint8).pin_memory()
    F_pinned.numpy()[...] = case.flags
    ecase = case.with_(T_init=T_pinned.numpy(), flags=F_pinned.numpy())
    out = [torch.empty((case.ny, case.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    ptrs = [C.cast(o.data_ptr(), C.POINTER(C.c_double)) for o in out]
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t = [time.perf_counter()]
    p, keep = P.make_params(ecase, storage)
    need = L.lbm_footprint_bytes(C.byref(p))
    if need == 0:
        raise RuntimeError(L.lbm_last_error(None).decode())
    t.append(time.perf_counter())
    mem = torch.empty(int(need), dtype=torch.uint8, device="cuda")
    h = C.c_void_p()
    st = L.lbm_create(C.byref(p), C.c_void_p(stream.cuda_stream), C.c_void_p(mem.data_ptr()), C.c_size_t(need),
                      C.byref(h))
    if st != 0:
        raise RuntimeError(L.lbm_last_error(None).decode())
    t.append(time.perf_counter())
    st = L.lbm_step(h, C.c_int64(steps))
    if st == 0:
        st = L.lbm_sync(h)
    t.append(time.perf_counter())
    if st == 0:
        st = L.lbm_read_macro(h, *ptrs)
    if st != 0:
        raise RuntimeError(L.lbm_last_error(h).decode())
    t.append(time.perf_counter())
    L.lbm_destroy(h)
    del mem
    t.append(time.perf_counter())
    del keep
    h2d = case.nx * case.ny * (8 + 1)  # T_init + flags
    d2h = 4 * 8 * case.nx * case.ny    # rho, ux, uy, T
    names = ("footprint", "create", "steps", "read_macro", "destroy")
    phases = {n: round((t[k + 1] - t[k]) * 1e3, 3) for k, n in enumerate(names)}
    rates = {"create_h2d_GBps": round(h2d / ((t[2] - t[1]) * 1e9), 1),
             "read_d2h_GBps": round(d2h / ((t[4] - t[3]) * 1e9), 1)}
    return (t[-1] - t[0]), h2d, d2h, phases, rates


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
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores,
    on the same workload (the full --nx x --H Rayleigh-Benard cell): each bench
    step is one oracle step over the whole lattice (about 70 ms on 16 cores for
    4096 x 2048), so that --steps 20 --warmup 5 ends within seconds."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    nx, H = args.nx, args.H
    case = workload(nx, H)
    threads = min(os.cpu_count() or 1, oracle.threads_available())
    o = oracle.OracleLattice(case, threads=threads)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = case.fluid_nodes * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"rayleigh_benard_{nx}x{H}_ra1e6", "nx": nx, "ny": H, "storage": "f64 (CPU oracle)",
                   "sample": f"each step: one oracle step over the whole {nx}x{H} lattice"},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": f"the whole {nx}x{H} workload, {args.steps} steps after {args.warmup}, "
                                   f"{dt:.2f} s, OpenMP over rows"},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def set_member_kernel(b, code: int):
    """The concurrent kind's member kernel from the tuner's code: -1 the members'
    own, 0-4 VEC4 at that config, 5-9 VEC4W at config - 5."""
    if code < 0:
        b.set_member_kernel("auto", 0)
    else:
        b.set_member_kernel("vec4" if code < 5 else "vec4w", code % 5)


def run_batched(args):
    """Batched uneven lattices: `--count` differentially heated cavities, sides
    uniform over 128..1024, Ra log-uniform in [1e3, 1e6], advanced together.
    The autotuner times every kind and config; each kind is then timed on its
    best config with CUDA-graph replay, and the tuned choice runs the full
    `--steps` (5e4 for the stated workload), device-timed. Also: every member
    stepped with its own launches, one after another."""
    import torch
    import paper_1510_08224_gb300 as P
    torch.cuda.set_device(0)
    if args.batch_members == "rb":
        # `--count` copies of the benchmark lattice (--nx x --H): with --count 1 the batch
        # kernels run on exactly the single-lattice kernel's shape, which isolates their
        # per-kernel cost from the narrow members of the cavity mix
        cases = [workload(args.nx, args.H) for _ in range(args.count)]
        wl = f"batched_rayleigh_benard_{args.nx}x{args.H}_{args.count}"
    else:
        cases = lc.batched_cavities(count=args.count, seed=0)
        wl = f"batched_cavities_{args.count}"
    cells = sum(c.fluid_nodes for c in cases)
    stream = torch.cuda.current_stream()
    lats = [P.Lattice(c, storage=args.storage, stream=stream) for c in cases]
    b = P.Batch(stream=stream)
    for lat in lats:
        b.add(lat)
    b.step(args.warmup)
    if args.no_tune:
        # one kind and config (profiling): --batch-kind, --config, graphs of 32 steps
        b.set_kind(args.batch_kind)
        if args.batch_kind == "concurrent":
            # --config -1: the members' own kernels; 0-4: VEC4 at that config; 5-9: VEC4W at config - 5
            set_member_kernel(b, args.config)
        else:
            b.set_config(args.config, args.rows_per_unit)
        b.set_mode(32, 32)
        b.step(args.warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        b.close()
        peak, _ = measured_peak()
        print(json.dumps({"workload": wl, "storage": args.storage,
                          "kind": args.batch_kind, "config": args.config, "rows_per_unit": args.rows_per_unit,
                          "steps": args.steps,
                          "fluid_cells": cells, "ms_per_step": round(ms, 5),
                          "MLUPS": round(cells / (ms * 1e-3) / 1e6, 1),
                          "frac": round(BYTES_PER_NODE[args.storage] * cells / (ms * 1e-3) / 1e9 / peak, 4)}),
              flush=True)
        return 0
    tuned_kind, tuned_cfg, ms_cand = b.tune(trial_steps=64)
    tuned_unit = b.info()["rows_per_unit"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, steps, warm=args.warmup):
        fn(warm)
        torch.cuda.synchronize()
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    peak, peak_src = measured_peak()
    bpn = BYTES_PER_NODE[args.storage]

    def rate(ms, steps):
        per = ms / steps
        return {"MLUPS": round(cells / (per * 1e-3) / 1e6, 1), "ms_per_step": round(per, 5),
                "frac": round(bpn * cells / (per * 1e-3) / 1e9 / peak, 4)}

    kinds = {}
    k_steps = min(args.steps, 2000)
    for kind in ("fused", "persistent", "concurrent"):
        b.set_kind(kind)
        if kind == "concurrent":
            cands = {-1: ms_cand["concurrent"]}
            cands.update({c: ms_cand[f"concurrent_vec4_cfg{c}"] for c in range(5)})
            cands.update({5 + c: ms_cand[f"concurrent_vec4w_cfg{c}"] for c in range(5)})
            cfg = min(cands, key=cands.get)
            set_member_kernel(b, cfg)
        elif kind == "fused":
            cands = {c: ms_cand[f"fused_cfg{c}"] for c in range(10)}
            cfg = min(cands, key=cands.get)
            b.set_config(cfg, 1)
        else:
            cands = {(c, 1): ms_cand[f"persistent_cfg{c}"] for c in range(5)}
            cands.update({(c, 2): ms_cand[f"persistent_u2_cfg{c}"] for c in range(5)})
            cfg, unit = min(cands, key=cands.get)
            b.set_config(cfg, unit)
        b.set_mode(32, 32)
        kinds[kind] = {"config": cfg, **rate(timed(b.step, k_steps), k_steps)}
        if kind == "persistent":
            kinds[kind]["rows_per_unit"] = unit
        if kind == "concurrent":
            kinds[kind]["member_kernel"] = list(b.get_member_kernel())
    # the tuned choice over the full run
    b.set_kind(tuned_kind)
    if tuned_kind == "concurrent":
        set_member_kernel(b, tuned_cfg)
    else:
        b.set_config(tuned_cfg, tuned_unit if tuned_kind == "persistent" else 1)
    b.set_mode(32, 32)
    member_kernel = list(b.get_member_kernel()) if tuned_kind == "concurrent" else None
    sampler = ClockSampler(0).start()
    t_start = time.perf_counter()
    ms = timed(b.step, args.steps)
    t_end = time.perf_counter()
    sampler.stop()
    launches_per_step = {"fused": 1, "persistent": 1 / 32, "concurrent": args.count}[tuned_kind]
    finite = True
    for lat in lats:
        try:
            lat.residual()
        except P.LBMError:
            finite = False
    b.close()

    def serial(n):
        for _ in range(n):
            for lat in lats:
                lat.step(1)
    k_serial = max(10, min(args.steps, 2000) // 10)
    ms_serial = timed(serial, k_serial)
    tuned = rate(ms, args.steps)
    value = tuned["MLUPS"]
    kernel = {"fused": "k_batch_grid_w" if tuned_cfg >= 5 else "k_batch_grid", "persistent": "k_batch_persistent",
              "concurrent": "each member's step kernel, concurrent streams"}[tuned_kind]
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tuned["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": COMPUTE_DTYPE[args.storage], "data": "synthetic",
        "config": {"workload": wl, "lattices": args.count, "fluid_cells": cells,
                   **({"sides": "uniform 128..1024", "Ra": "log-uniform [1e3, 1e6]"}
                      if args.batch_members == "cavities" else {"shape": f"{args.nx} x {args.H}", "Ra": 1e6}),
                   "storage": STORAGE_NAME[args.storage],
                   "tuned": {"kind": tuned_kind, "config": tuned_cfg, "member_kernel": member_kernel,
                             "rows_per_unit": tuned_unit if tuned_kind == "persistent" else None, "graph_steps": 32,
                             "steps_per_launch": 32 if tuned_kind == "persistent" else 1},
                   "l2": "no flush: working set > L2",
                   "tune_ms_per_step": {k: (round(m, 5) if np.isfinite(m) else None) for k, m in ms_cand.items()}},
        "kinds": kinds,
        "finite": finite,
        "serial_per_lattice": {**rate(ms_serial, k_serial), "steps": k_serial, "launches_per_step": args.count},
        "roofline": {"bound": "hbm", "achieved": round(bpn * cells / (tuned["ms_per_step"] * 1e-3) / 1e9, 1),
                     "peak": peak, "unit": "GB/s", "frac": tuned["frac"], "traffic": None, "kernel": kernel,
                     "bytes_per_node": bpn, "peak_source": f"{peak_src} HBM copy bandwidth (burst)"},
        "gpu_launches": int(round(args.steps * launches_per_step)),
        "clocks": sampler.summary(t_start, t_end),
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
                kernels += [("scalar", 0)] + [(v, c) for v in ("vec4", "vec4w")
                                              for c in range(P.step_kernel_count(st, v))]
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
                row[f"{v[0]}{v[1] if v[0] in ('vec4', 'vec4w') else ''}"] = {
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


# Rayleigh-Benard requests are drawn from the band of stationary convection rolls: below
# onset (Ra ~ 1708) the flow decays at a constant relative rate, so the relative residual of u
# never falls; above a few 1e4 the 2-D cell is time-dependent (measured: of the cells of sides
# 32-256 at Ra 1e3 / 1e4 / 1e5 / 1e6, 0 / 7 / 2 / 1 of 7 reached R < 1e-6 within 6e5 steps)
RB_STEADY_RA = (2e3, 2e4)


def serving_measure(storage: str, count: int, side_lo: int, side_hi: int, step_cap: int, check_every: int,
                    graph_steps: int, rate: float, budget_frac: float | None, kind: str, cavity_share: float,
                    ra_lo: float = 1e3, ra_hi: float = 1e6, rb_ra=RB_STEADY_RA, batch_config: int = -1):
    """Continuous-batching serving against the plain path, on the same seeded
    stream: Poisson arrivals (`rate` per second, seed 0) of `count` cavity (a
    share `cavity_share`) and Rayleigh-Benard requests, sides log-uniform in
    [side_lo, side_hi], Ra log-uniform in [ra_lo, ra_hi] (Rayleigh-Benard cells: in
    the band of steady rolls, RB_STEADY_RA), each run to residual
    < 1e-6 (checked every `check_every` steps) or the step cap. Served: every
    admitted request resident in FP32/FP16 storage, stepped together by one
    batch (`kind`), residuals of all read with one synchronisation, admitted
    first come first served while its footprint fits the HBM budget (150 GB, or
    `budget_frac` of the stream's total footprint so that admission binds).
    Plain: FP64 storage, one request at a time with its own launches, through
    the same real-time loop. Returns (config, served, plain)."""
    import torch
    from paper_1510_08224_gb300 import serve
    torch.cuda.set_device(0)
    stream = lc.serving_stream(n=count, seed=0, side_lo=side_lo, side_hi=side_hi, rate=rate, ra_lo=ra_lo,
                               ra_hi=ra_hi, cavity_share=cavity_share, rb_ra=rb_ra)
    reqs = [serve.Request(k, c, t, nusselt_sides=((0,) if kind_ == "cavity" else (2,))) for k, (t, kind_, c) in
            enumerate(stream)]
    cells = sum(int((r.case.flags == 0).sum()) for r in reqs)
    be = serve.GpuBackend(storage, graph_steps=graph_steps, kind=kind, config=batch_config)
    total_fp = sum(be.footprint(r.case) for r in reqs)
    budget = 150e9 if budget_frac is None else max(budget_frac * total_fp,
                                                   max(be.footprint(r.case) for r in reqs))
    srv = serve.Server(be, budget_bytes=budget, check_every=check_every, tol=1e-6, step_cap=step_cap)
    t0 = time.perf_counter()
    res = srv.run(reqs, realtime=True)
    span = time.perf_counter() - t0
    be.close()
    pb = serve.PlainBackend("f64")
    psrv = serve.Server(pb, budget_bytes=150e9, check_every=check_every, tol=1e-6, step_cap=step_cap, max_active=1)
    t0 = time.perf_counter()
    base = psrv.run(reqs, realtime=True)
    pspan = time.perf_counter() - t0
    pb.close()
    same_steps = sum(1 for a, b in zip(sorted(res, key=lambda r: r.rid), sorted(base, key=lambda r: r.rid))
                     if a.steps == b.steps)
    config = {"workload": f"serving_stream_{count}", "arrivals": f"Poisson {rate:g}/s, seed 0",
              "sides": f"log-uniform [{side_lo}, {side_hi}]",
              "Ra": f"log-uniform [{ra_lo:g}, {ra_hi:g}] (cavities), [{rb_ra[0]:g}, {rb_ra[1]:g}] (Rayleigh-Benard)",
              "types": f"cavity {cavity_share:g} | rayleigh_benard {1 - cavity_share:g}", "tol": 1e-6,
              "step_cap": srv.step_cap, "check_every": check_every, "hbm_budget_bytes": budget,
              "total_footprint_bytes": total_fp, "storage": STORAGE_NAME[storage], "batch_kind": kind,
              "batch_config": batch_config,
              "requests": len(reqs), "fluid_cells_total": cells, "graph_steps": graph_steps}
    served = {**serve.summarize(res, span), **serve.summarize_converged(res), "makespan_s": round(span, 3),
              "peak_hbm_bytes": srv.peak_in_use, "max_concurrent": srv.max_active,
              "queued_for_memory": srv.queued_for_memory, "MLUPS": round(sum(r.cells * r.steps for r in res) /
                                                                          span / 1e6, 1)}
    plain = {**serve.summarize(base, pspan), **serve.summarize_converged(base), "makespan_s": round(pspan, 3),
             "MLUPS": round(sum(r.cells * r.steps for r in base) / pspan / 1e6, 1), "same_step_counts": same_steps,
             "what": "FP64 storage, one request at a time (max_active 1), real-time run of the same stream"}
    return config, served, plain


def run_serving(args):
    """The serving stream as its own bench line (value = solves/s)."""
    config, served, plain = serving_measure(args.storage, args.count, args.side_lo, args.side_hi, args.step_cap,
                                            args.check_every, args.graph_steps, args.rate, args.budget_frac,
                                            args.batch_kind, args.cavity_share, batch_config=args.batch_config)
    line = {
        "metric": METRIC, "value": round(served["solves_per_s"], 4), "unit": "solves/s", "n_gpus": 1,
        "steps": config["step_cap"], "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": COMPUTE_DTYPE[args.storage], "data": "synthetic", "config": config,
        "served": served, "plain_fp64": plain,
        "speedup_solves_per_s": round(served["solves_per_s"] / plain["solves_per_s"], 2),
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
    ap.add_argument("--variant", default="auto", choices=["auto", "scalar", "vec4", "vec4w", "vec8", "tma"],
                    help="step kernel variant (lbm_set_step_kernel)")
    ap.add_argument("--config", type=int, default=0, help="shape index of the step variant")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="rb: skip the short serving stream")
    ap.add_argument("--no-tune", action="store_true",
                    help="batch: run --batch-kind at --config only (no tuner, no sweep of kinds): for profiling")
    ap.add_argument("--sweep", action="store_true", help="cost workload: time every step kernel of each model")
    ap.add_argument("--workload", default="rb", choices=["rb", "batch", "serve", "cost", "table3"],
                    help="rb: the 4096 x 2048 Rayleigh-Benard step (default); batch: uneven cavities advanced together; serve: the serving stream; cost: collision operators; table3: the cavity of Table 3")
    ap.add_argument("--count", type=int, default=64, help="lattices (batch) or requests (serve)")
    ap.add_argument("--side-lo", type=int, default=32, help="smallest side of a served request")
    ap.add_argument("--side-hi", type=int, default=128, help="largest side of a served request")
    ap.add_argument("--step-cap", type=int, default=300000, help="step cap of a served request")
    ap.add_argument("--check-every", type=int, default=500, help="steps between residual checks (serve)")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrival rate (requests per second)")
    ap.add_argument("--budget-frac", type=float, default=None,
                    help="serve: HBM budget as a fraction of the stream's total footprint (default: 150 GB)")
    ap.add_argument("--batch-members", default="cavities", choices=["cavities", "rb"],
                    help="batch: the uneven cavity mix, or --count copies of the --nx x --H lattice")
    ap.add_argument("--batch-config", type=int, default=-1,
                    help="serve: the batch's kernel config (lbm_batch_set_config; -1 the default)")
    ap.add_argument("--rows-per-unit", type=int, default=1,
                    help="batch --no-tune: row segments per work unit of the persistent kernel")
    ap.add_argument("--batch-kind", default="fused", choices=["fused", "persistent", "concurrent"],
                    help="serve: batch kind of the served path")
    ap.add_argument("--cavity-share", type=float, default=0.75, help="serve: share of cavity requests")
    ap.add_argument("--graph-steps", type=int, default=50,
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
    lat.residual()  # snapshot before the timed region: the check after it is a real residual
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
    r = lat.residual()  # residual over the timed steps: finite, or LBMError if the state diverged
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
    dfma = None
    if args.storage == "f64" or not args.no_variants:
        try:
            dfma = P.probe_fp64_rate()
        except P.LBMError:
            dfma = None
    if args.storage == "f64":
        alu = fp64_alu_roofline(value / world, dfma)
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
        e2e_run(P, torch, case, args.storage, e2e_steps)  # warm: first-use costs (allocator, graph capture)
        secs, h2d, d2h, phases, rates = e2e_run(P, torch, case, args.storage, e2e_steps)
        line["e2e"] = {"value": round(fluid * e2e_steps / secs / 1e6, 1), "unit": "MLUPS",
                       "h2d_bytes_per_step": int(h2d / e2e_steps), "d2h_bytes_per_step": int(d2h / e2e_steps),
                       "steps": e2e_steps, "ms_total": round(secs * 1e3, 3), "phases_ms": phases, **rates,
                       "host_link_GBps": host_link_gbs(torch),
                       "what": "lbm_footprint_bytes, lbm_create from pinned host flags+T_init, lbm_step(K), "
                               "lbm_read_macro to pinned host, lbm_destroy; wall clock, second of two runs"}
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
                var[STORAGE_NAME[st]]["alu"] = fp64_alu_roofline(vm, dfma)
        line["variants"] = var
    if dfma:
        line["fp64_rate_measured"] = {"dfma_per_s": round(dfma, 1), "tflops": round(2 * dfma / 1e12, 4),
                                      "nominal_tflops": FP64_NOMINAL_TFLOPS,
                                      "how": "lbm_probe_fp64_rate: independent DFMA chains, 8 blocks of 256 "
                                             "threads per SM, best of 5 CUDA-event timed launches"}
    if rank == 0 and world == 1 and not args.no_serving:
        # the metric's second half (solves/s, p50/p99 latency against the plain path) on
        # a shorter stream than --workload serve, so that the default run stays short
        try:
            config, served, plain = serving_measure(args.storage if args.storage != "f64" else "f32", 24, 32, 64,
                                                    200_000, 500, 50, 200.0, 0.5, "fused", 0.75)
            line["serving"] = {"config": config, "served": served, "plain_fp64": plain,
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
