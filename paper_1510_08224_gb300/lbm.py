"""ctypes binding of the C ABI in ``include/nomrt_lbm.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libnomrt_lbm.so``. PyTorch supplies device memory and the stream.
There is no CPU fallback: if the library cannot be built or loaded, importing
the binding's functions raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EDIVERGED, LBM_ETIMEOUT = range(6)
STORAGE = {"f64": 0, "f32": 1, "f16": 2}
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16": 2}
SIDES = {"left": 0, "right": 1, "bottom": 2, "top": 3}

STEP_VARIANTS = {"auto": 0, "scalar": 1, "vec4": 2, "tma": 3, "vec8": 4, "vec4w": 5}
# Every symbol include/nomrt_lbm.h declares.
EXPORTED = ("lbm_footprint_bytes", "lbm_validate", "lbm_create", "lbm_step", "lbm_sync", "lbm_step_kernel_count",
            "lbm_set_step_kernel", "lbm_read_macro", "lbm_read_macro_rows",
            "lbm_nusselt",
            "lbm_residual", "lbm_get_populations", "lbm_set_populations", "lbm_info", "lbm_last_error",
            "lbm_destroy", "lbm_residual_fields_noalloc", "lbm_probe_fp64_rate", "lbm_bounds_checking",
            "lbm_debug_bounds_limit", "lbm_batch_create", "lbm_batch_add", "lbm_batch_remove",
            "lbm_batch_set_mode", "lbm_batch_set_kind", "lbm_batch_set_config", "lbm_batch_tune", "lbm_batch_step", "lbm_batch_sync",
            "lbm_batch_info", "lbm_batch_get_mode", "lbm_batch_residuals", "lbm_batch_last_error", "lbm_batch_destroy",
            "lbm_batch_debug_barrier_extra", "lbm_batch_set_member_kernel", "lbm_batch_get_member_kernel")
BATCH_KINDS = {"fused": 0, "concurrent": 1, "persistent": 2}


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lbm status {status}: {msg}")
        self.status = status


class lbm_wall(C.Structure):
    _fields_ = [("ux", C.c_double), ("uy", C.c_double), ("kind", C.c_int32), ("scheme", C.c_int32),
                ("T", C.c_double)]


class lbm_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("periodic_x", C.c_int32), ("periodic_y", C.c_int32),
        ("flags", C.c_void_p), ("walls", C.c_void_p), ("n_walls", C.c_int32), ("storage", C.c_int32),
        ("nu", C.c_double), ("alpha", C.c_double), ("g_beta", C.c_double), ("T0", C.c_double),
        ("ax", C.c_double), ("ay", C.c_double),
        ("s_e", C.c_double), ("s_q", C.c_double), ("s_eps", C.c_double),
        ("zeta_e", C.c_double), ("zeta_nu", C.c_double), ("varpi", C.c_double),
        ("T_init", C.c_void_p),
        ("thermal_q", C.c_int32), ("theta", C.c_double),
        ("zeta_q", C.c_double), ("zeta_eps", C.c_double),
        ("collision", C.c_int32),
    ]


_lib = None
_lock = threading.Lock()


def library_variant() -> str:
    """'' for the library, 'bounds' for the bounds-checking build, chosen by the
    environment variable NOMRT_LIB_VARIANT when the library is first loaded."""
    v = os.environ.get("NOMRT_LIB_VARIANT", "")
    if v not in _build.VARIANTS:
        raise ValueError(f"NOMRT_LIB_VARIANT must be one of {sorted(_build.VARIANTS)}")
    return v


def library_path() -> str:
    return _build.library_path(library_variant())


def load():
    """Build (if stale) and load the CUDA library. Raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build(variants=(library_variant(),))
        L = C.CDLL(path)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.lbm_footprint_bytes.restype = C.c_size_t
        L.lbm_footprint_bytes.argtypes = [C.POINTER(lbm_params)]
        L.lbm_validate.restype = C.c_int
        L.lbm_validate.argtypes = [C.POINTER(lbm_params)]
        L.lbm_create.restype = C.c_int
        L.lbm_create.argtypes = [C.POINTER(lbm_params), vp, vp, C.c_size_t, C.POINTER(vp)]
        L.lbm_step.restype = C.c_int
        L.lbm_step.argtypes = [vp, C.c_int64]
        L.lbm_sync.restype = C.c_int
        L.lbm_sync.argtypes = [vp]
        L.lbm_step_kernel_count.restype = C.c_int32
        L.lbm_step_kernel_count.argtypes = [C.c_int32, C.c_int32]
        L.lbm_set_step_kernel.restype = C.c_int
        L.lbm_set_step_kernel.argtypes = [vp, C.c_int32, C.c_int32]
        L.lbm_read_macro.restype = C.c_int
        L.lbm_read_macro.argtypes = [vp, dp, dp, dp, dp]
        L.lbm_read_macro_rows.restype = C.c_int
        L.lbm_read_macro_rows.argtypes = [vp, C.c_int32, C.c_int32, dp, dp, dp, dp]
        L.lbm_nusselt.restype = C.c_int
        L.lbm_nusselt.argtypes = [vp, C.c_int32, C.c_double, C.c_double, dp]
        L.lbm_residual.restype = C.c_int
        L.lbm_residual.argtypes = [vp, dp]
        L.lbm_get_populations.restype = C.c_int
        L.lbm_get_populations.argtypes = [vp, dp, dp]
        L.lbm_set_populations.restype = C.c_int
        L.lbm_set_populations.argtypes = [vp, dp, dp]
        L.lbm_info.restype = C.c_int
        L.lbm_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int64)]
        L.lbm_last_error.restype = C.c_char_p
        L.lbm_last_error.argtypes = [vp]
        L.lbm_destroy.restype = None
        L.lbm_destroy.argtypes = [vp]
        for name, args in (("lbm_batch_create", [vp, C.POINTER(vp)]), ("lbm_batch_add", [vp, vp]),
                           ("lbm_batch_remove", [vp, vp]), ("lbm_batch_set_mode", [vp, C.c_int32, C.c_int32]),
                           ("lbm_batch_set_config", [vp, C.c_int32, C.c_int32]), ("lbm_batch_set_kind", [vp, C.c_int32]),
                           ("lbm_batch_tune", [vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                               C.POINTER(C.c_float)]),
                           ("lbm_batch_get_mode", [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                                   C.POINTER(C.c_int32)]),
                           ("lbm_batch_residuals", [vp, C.c_int32, C.POINTER(vp), dp, C.POINTER(C.c_int32)]),
                           ("lbm_batch_step", [vp, C.c_int64]), ("lbm_batch_sync", [vp]),
                           ("lbm_batch_debug_barrier_extra", [vp, C.c_int32]),
                           ("lbm_batch_set_member_kernel", [vp, C.c_int32, C.c_int32]),
                           ("lbm_batch_get_member_kernel", [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
                           ("lbm_batch_info", [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                               C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64)])):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = args
        L.lbm_batch_last_error.restype = C.c_char_p
        L.lbm_batch_last_error.argtypes = [vp]
        L.lbm_batch_destroy.restype = None
        L.lbm_batch_destroy.argtypes = [vp]
        L.lbm_bounds_checking.restype = C.c_int32
        L.lbm_bounds_checking.argtypes = []
        L.lbm_debug_bounds_limit.restype = C.c_int
        L.lbm_debug_bounds_limit.argtypes = [vp, C.c_int64]
        L.lbm_probe_fp64_rate.restype = C.c_int
        L.lbm_probe_fp64_rate.argtypes = [vp, dp]
        L.lbm_residual_fields_noalloc.restype = C.c_int
        L.lbm_residual_fields_noalloc.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.c_int64, vp, dp]
        _lib = L
        return L


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(status: int, handle=None):
    if status != LBM_OK:
        msg = load().lbm_last_error(handle)
        raise LBMError(status, msg.decode() if msg else "")


def make_params(case, storage: str = "f32"):
    """lbm_params from any object with the problem's attributes (nx, ny,
    periodic_x, periodic_y, flags, walls, nu, alpha, g_beta, T0, ax, ay, s_e,
    s_q, s_eps, zeta_e, zeta_nu, varpi, T_init; optionally thermal_q, theta,
    zeta_q, zeta_eps for the D2Q9 temperature model and collision, 1 for BGK).
    Returns (params, keepalive)."""
    flags = np.ascontiguousarray(case.flags, dtype=np.uint8)
    assert flags.shape == (case.ny, case.nx)
    walls = (lbm_wall * max(1, len(case.walls)))()
    for k, w in enumerate(case.walls):
        walls[k] = lbm_wall(float(w.ux), float(w.uy), int(w.kind), int(getattr(w, "scheme", 0)), float(w.T))
    Ti = None
    if getattr(case, "T_init", None) is not None:
        Ti = np.ascontiguousarray(case.T_init, dtype=np.float64)
        assert Ti.shape == (case.ny, case.nx)
    p = lbm_params()
    p.nx, p.ny = int(case.nx), int(case.ny)
    p.periodic_x, p.periodic_y = int(bool(case.periodic_x)), int(bool(case.periodic_y))
    p.flags = flags.ctypes.data
    p.walls = C.addressof(walls)
    p.n_walls = len(case.walls)
    p.storage = STORAGE[storage]
    for name in ("nu", "alpha", "g_beta", "T0", "ax", "ay", "s_e", "s_q", "s_eps", "zeta_e", "zeta_nu", "varpi"):
        setattr(p, name, float(getattr(case, name)))
    p.T_init = Ti.ctypes.data if Ti is not None else None
    p.thermal_q = int(getattr(case, "thermal_q", 5))
    p.theta = float(getattr(case, "theta", 1.0))
    p.zeta_q = float(getattr(case, "zeta_q", 1.0))
    p.zeta_eps = float(getattr(case, "zeta_eps", 1.0))
    p.collision = int(getattr(case, "collision", 0))
    return p, (flags, walls, Ti)


def residual_fields_noalloc(ux, uy, T, ux_prev, uy_prev, T_prev, solid=None, stream=None) -> float:
    """lbm_residual_fields_noalloc on torch CUDA tensors (float64, same length;
    solid: uint8 or None). Allocates nothing on the device."""
    import torch
    n = ux.numel()
    fields = (ux, uy, T, ux_prev, uy_prev, T_prev)
    for a in fields:
        if not isinstance(a, torch.Tensor) or not a.is_cuda or a.dtype != torch.float64:
            raise TypeError("fields must be float64 CUDA tensors")
        if not a.is_contiguous() or a.numel() != n or a.device != ux.device:
            raise ValueError("fields must be contiguous, of one length and on one device")
    if solid is not None:
        if not isinstance(solid, torch.Tensor) or not solid.is_cuda or solid.dtype != torch.uint8:
            raise TypeError("solid must be a uint8 CUDA tensor or None")
        if not solid.is_contiguous() or solid.numel() != n or solid.device != ux.device:
            raise ValueError("solid must be contiguous, of the fields' length and on their device")
    st = stream if stream is not None else torch.cuda.current_stream(ux.device)
    r = C.c_double()
    with torch.cuda.device(ux.device):
        status = load().lbm_residual_fields_noalloc(
            ux.data_ptr(), uy.data_ptr(), T.data_ptr(), ux_prev.data_ptr(), uy_prev.data_ptr(), T_prev.data_ptr(),
            None if solid is None else solid.data_ptr(), C.c_int64(n), C.c_void_p(st.cuda_stream), C.byref(r))
    _check(status, None)
    return r.value


def probe_fp64_rate(stream=None) -> float:
    """The current device's FP64 fused multiply-add rate (instructions per
    second; lbm_probe_fp64_rate)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    v = C.c_double()
    _check(load().lbm_probe_fp64_rate(C.c_void_p(st.cuda_stream), C.byref(v)), None)
    return v.value


def step_kernel_count(storage: str, variant) -> int:
    v = STEP_VARIANTS[variant] if isinstance(variant, str) else int(variant)
    return int(load().lbm_step_kernel_count(STORAGE[storage], v))


def step_kernels(storage: str):
    """Every (variant, config) pair available for a storage."""
    return [(v, c) for v in ("scalar", "vec4", "vec4w", "vec8", "tma") for c in range(step_kernel_count(storage, v))]


def lbm_footprint_bytes(params) -> int:
    return int(load().lbm_footprint_bytes(C.byref(params)))


def validate(case, storage: str = "f32") -> None:
    """Every check lbm_create makes (lbm_validate, host only); raises LBMError
    naming the first invalid cell."""
    p, keep = make_params(case, storage)
    st = load().lbm_validate(C.byref(p))
    if st != LBM_OK:
        raise LBMError(st, load().lbm_last_error(None).decode())


class Lattice:
    """A lattice resident on the GPU. Device memory is a torch uint8 tensor
    (``device_mem="torch"``, the default) or allocated by the library
    (``device_mem="library"``); work is queued on ``stream`` (a
    ``torch.cuda.Stream``; default: the current stream)."""

    def __init__(self, case, storage: str = "f32", stream=None, device_mem: str = "torch", device=None):
        import torch

        L = load()
        self.case = case
        self.storage = storage
        self.nx, self.ny = int(case.nx), int(case.ny)
        self.tq = 9 if int(getattr(case, "thermal_q", 5)) == 9 else 5
        p, keep = make_params(case, storage)
        need = L.lbm_footprint_bytes(C.byref(p))
        if need == 0:
            raise LBMError(LBM_EINVAL, L.lbm_last_error(None).decode())
        self.footprint = int(need)
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._mem = None
        mem_ptr, mem_bytes = None, 0
        if device_mem == "torch":
            self._mem = torch.empty(int(need), dtype=torch.uint8, device=dev)
            mem_ptr, mem_bytes = self._mem.data_ptr(), int(need)
        elif device_mem != "library":
            raise ValueError("device_mem must be 'torch' or 'library'")
        h = C.c_void_p()
        with torch.cuda.device(dev):
            st = L.lbm_create(C.byref(p), C.c_void_p(self._stream.cuda_stream), C.c_void_p(mem_ptr),
                              C.c_size_t(mem_bytes), C.byref(h))
        _check(st, None)
        self._h = h
        del keep

    # -- lifetime
    def close(self):
        h = getattr(self, "_h", None)
        if h:
            load().lbm_destroy(h)
            self._h = None
        self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- calls
    def step(self, n: int = 1):
        _check(load().lbm_step(self._h, int(n)), self._h)

    def sync(self):
        _check(load().lbm_sync(self._h), self._h)

    def set_step_kernel(self, variant, config: int = 0):
        """variant 'auto', 'scalar', 'vec4', 'vec4w', 'vec8' or 'tma' and a config index
        (see lbm_set_step_kernel)."""
        v = STEP_VARIANTS[variant] if isinstance(variant, str) else int(variant)
        _check(load().lbm_set_step_kernel(self._h, v, int(config)), self._h)
        self.kernel = (variant, int(config))

    def macro(self):
        """(rho, ux, uy, T), each (ny, nx) float64 on the host."""
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        _check(load().lbm_read_macro(self._h, *[_dptr(a) for a in out]), self._h)
        return tuple(out)

    def macro_rows(self, y0: int, y1: int):
        """(rho, ux, uy, T) of rows y0 <= y < y1, each (y1 - y0, nx) float64."""
        out = [np.empty((max(0, y1 - y0), self.nx)) for _ in range(4)]
        _check(load().lbm_read_macro_rows(self._h, int(y0), int(y1), *[_dptr(a) for a in out]), self._h)
        return tuple(out)

    def nusselt(self, side, L: float = 0.0, delta_T: float = 1.0) -> float:
        side = SIDES[side] if isinstance(side, str) else int(side)
        v = C.c_double()
        _check(load().lbm_nusselt(self._h, side, float(L), float(delta_T), C.byref(v)), self._h)
        return v.value

    def residual(self) -> float:
        v = C.c_double()
        _check(load().lbm_residual(self._h, C.byref(v)), self._h)
        return v.value

    def populations(self):
        f = np.empty((9, self.ny, self.nx)); g = np.empty((self.tq, self.ny, self.nx))
        _check(load().lbm_get_populations(self._h, _dptr(f), _dptr(g)), self._h)
        return f, g

    def set_populations(self, f=None, g=None):
        f = None if f is None else np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        g = None if g is None else np.ascontiguousarray(g, dtype=np.float64).reshape(self.tq, self.ny, self.nx)
        _check(load().lbm_set_populations(self._h, _dptr(f), _dptr(g)), self._h)

    def info(self):
        fl, st = C.c_int64(), C.c_int64()
        pitch, eb = C.c_int32(), C.c_int32()
        _check(load().lbm_info(self._h, C.byref(fl), C.byref(pitch), C.byref(eb), C.byref(st)), self._h)
        return dict(fluid_cells=fl.value, pitch=pitch.value, elem_bytes=eb.value, steps=st.value)


class Batch:
    """Lattices of uneven size advanced together (see the lbm_batch_* calls).
    Members must share the batch's stream and one of the FP32/FP16 storages."""

    def __init__(self, stream=None):
        import torch
        L = load()
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        st = L.lbm_batch_create(C.c_void_p(self._stream.cuda_stream), C.byref(h))
        if st != LBM_OK:
            raise LBMError(st, L.lbm_last_error(None).decode())
        self._h = h
        self.members = []

    def _check(self, st):
        if st != LBM_OK:
            raise LBMError(st, load().lbm_batch_last_error(self._h).decode())

    @property
    def stream(self):
        return self._stream

    def add(self, lat: "Lattice"):
        self._check(load().lbm_batch_add(self._h, lat.handle))
        self.members.append(lat)

    def remove(self, lat: "Lattice"):
        self._check(load().lbm_batch_remove(self._h, lat.handle))
        self.members.remove(lat)

    def set_mode(self, steps_per_launch: int = 32, graph_steps: int = 32):
        """Steps per launch of the persistent kind, and steps per replayed CUDA
        graph (0: launches from the host)."""
        self._check(load().lbm_batch_set_mode(self._h, int(steps_per_launch), int(graph_steps)))

    def get_mode(self):
        """(kind name, steps per launch, graph steps) in force."""
        k, spl, gs = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(load().lbm_batch_get_mode(self._h, C.byref(k), C.byref(spl), C.byref(gs)))
        names = {v: n for n, v in BATCH_KINDS.items()}
        return names[k.value], spl.value, gs.value

    def set_kind(self, kind):
        """'fused' (one launch per step over every member's rows), 'persistent'
        (one cooperative launch per steps_per_launch steps, grid barrier between
        steps) or 'concurrent' (a single-lattice kernel per member, side by side)."""
        k = BATCH_KINDS[kind] if isinstance(kind, str) else int(kind)
        self._check(load().lbm_batch_set_kind(self._h, k))

    def set_config(self, config: int, rows_per_unit: int = 1):
        self._check(load().lbm_batch_set_config(self._h, int(config), int(rows_per_unit)))

    def set_member_kernel(self, variant="auto", config: int = 0):
        """The step kernel every member runs in the concurrent kind: 'auto'
        (each member's own choice), 'scalar', or 'vec4' / 'vec4w' with a
        config 0..4 (lbm_batch_set_member_kernel)."""
        v = STEP_VARIANTS[variant] if isinstance(variant, str) else int(variant)
        self._check(load().lbm_batch_set_member_kernel(self._h, v, int(config)))

    def get_member_kernel(self):
        """(variant name, config) of the concurrent kind's member kernel."""
        v, c = C.c_int32(), C.c_int32()
        self._check(load().lbm_batch_get_member_kernel(self._h, C.byref(v), C.byref(c)))
        names = {n: k for k, n in STEP_VARIANTS.items()}
        return names[v.value], c.value

    def tune(self, trial_steps: int = 8):
        """Autotune kind and config on the current members (state unchanged).
        Returns (kind name, config, {candidate: ms per step}) with candidates
        fused_cfg0-9 (5-9: one row segment per warp), persistent_cfg0-4 and
        persistent_u2_cfg0-4 (work units of two row segments; the unit size
        chosen is info()['rows_per_unit']),
        concurrent (the members' own kernels),
        concurrent_vec4_cfg0-4 and concurrent_vec4w_cfg0-4; for the concurrent
        kind the config is -1 (own), 0-4 (vec4) or 5-9 (vec4w), already in
        force as the member kernel."""
        kind, cfg = C.c_int32(), C.c_int32()
        ms = (C.c_float * 31)()
        self._check(load().lbm_batch_tune(self._h, int(trial_steps), C.byref(kind), C.byref(cfg), ms))
        table = {f"fused_cfg{c}": ms[c] for c in range(10)}
        table.update({f"persistent_cfg{c}": ms[10 + c] for c in range(5)})
        table.update({f"persistent_u2_cfg{c}": ms[15 + c] for c in range(5)})
        table["concurrent"] = ms[20]
        table.update({f"concurrent_vec4_cfg{c}": ms[21 + c] for c in range(5)})
        table.update({f"concurrent_vec4w_cfg{c}": ms[26 + c] for c in range(5)})
        names = {v: n for n, v in BATCH_KINDS.items()}
        return names[kind.value], cfg.value, table

    def step(self, n: int = 1):
        self._check(load().lbm_batch_step(self._h, int(n)))

    def residuals(self):
        """{Lattice: R} for every member (lbm_batch_residuals: one
        synchronisation; NaN for a member whose fields are not finite)."""
        m = len(self.members)
        hs = (C.c_void_p * max(1, m))()
        r = (C.c_double * max(1, m))()
        n = C.c_int32()
        self._check(load().lbm_batch_residuals(self._h, m, hs, r, C.byref(n)))
        by_handle = {lat.handle.value: lat for lat in self.members}
        return {by_handle[hs[i]]: r[i] for i in range(n.value)}

    def debug_barrier_extra(self, extra: int):
        """Test hook: make the persistent kernel's grid barrier time out (see
        lbm_batch_debug_barrier_extra)."""
        self._check(load().lbm_batch_debug_barrier_extra(self._h, int(extra)))

    def sync(self):
        self._check(load().lbm_batch_sync(self._h))

    def info(self):
        m, u, cfg, rows = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        cells, steps = C.c_int64(), C.c_int64()
        self._check(load().lbm_batch_info(self._h, C.byref(m), C.byref(cells), C.byref(u), C.byref(cfg),
                                          C.byref(rows), C.byref(steps)))
        return dict(members=m.value, cells=cells.value, units=u.value, config=cfg.value, rows_per_unit=rows.value,
                    steps=steps.value)

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            load().lbm_batch_destroy(h)
            self._h = None
        self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
