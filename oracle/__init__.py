"""Plain FP64 CPU oracle for the non-orthogonal MRT lattice Boltzmann method.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
(``paper_1510_08224_gb300``) never does, and the oracle imports nothing from it.

The arithmetic lives in ``nomrt_oracle.c`` (plain C, dense products with the
paper's printed matrices: Eq. 13, Eq. 26, Eqs. A1-A2). This module compiles it
with gcc on first use (or via :func:`build`) and wraps it with ctypes.

Pins: ``tests/test_oracle_pins.py`` checks every function here against what the
paper and the mathematics fix (closed forms, invariants, special cases, brute
force). Functions without a pin are marked "parity unpinned" in their docstring.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nomrt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction, OpenMP over rows)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("periodic_x", C.c_int32), ("periodic_y", C.c_int32),
        ("flags", C.c_void_p),
        ("n_walls", C.c_int32),
        ("wall_u", C.c_void_p), ("wall_kind", C.c_void_p), ("wall_T", C.c_void_p),
        ("nu", C.c_double), ("alpha", C.c_double),
        ("g_beta", C.c_double), ("T0", C.c_double),
        ("ax", C.c_double), ("ay", C.c_double),
        ("s_e", C.c_double), ("s_q", C.c_double), ("s_eps", C.c_double),
        ("zeta_e", C.c_double), ("zeta_nu", C.c_double), ("varpi", C.c_double),
        ("s8_literal", C.c_int32),
        ("T_init", C.c_void_p),
        ("wall_scheme", C.c_void_p),
        ("thermal_q", C.c_int32),
        ("theta", C.c_double),
        ("zeta_q", C.c_double), ("zeta_eps", C.c_double),
        ("collision", C.c_int32),
        ("rho_in_u_terms", C.c_int32),
        ("nee_uf_variant", C.c_int32),
    ]


class OrcRates(C.Structure):
    _fields_ = [
        ("s", C.c_double * 9), ("z", C.c_double * 9),
        ("g_beta", C.c_double), ("T0", C.c_double),
        ("ax", C.c_double), ("ay", C.c_double), ("varpi", C.c_double),
        ("s8_literal", C.c_int32), ("tq", C.c_int32), ("theta", C.c_double),
        ("bgk", C.c_int32), ("rho_in_u", C.c_int32),
    ]


def lib():
    """The compiled oracle. NOMRT_ORACLE_LIB, if set, names another build of
    the same source to load instead (the mutation tests plant a mistake in a
    copy of the source and check that the pins catch it)."""
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(os.environ.get("NOMRT_ORACLE_LIB") or build())
            dp = C.POINTER(C.c_double)
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(OrcParams)]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_step.argtypes = [C.c_void_p, C.c_int64]
            L.orc_set_threads.argtypes = [C.c_void_p, C.c_int]
            L.orc_macro.argtypes = [C.c_void_p, dp, dp, dp, dp]
            L.orc_get_populations.argtypes = [C.c_void_p, dp, dp]
            L.orc_set_populations.argtypes = [C.c_void_p, dp, dp]
            L.orc_update_node.argtypes = [C.c_void_p, dp, dp, C.c_int, C.c_int, dp, dp]
            L.orc_update_node.restype = C.c_int
            L.orc_nusselt.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
            L.orc_nusselt.restype = C.c_double
            L.orc_residual.argtypes = [C.c_void_p]
            L.orc_residual.restype = C.c_double
            L.orc_collide_node.argtypes = [C.POINTER(OrcRates), dp, dp, dp, dp, dp]
            L.orc_rates_from_params.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcRates)]
            L.orc_get_rates.argtypes = [C.c_void_p, C.POINTER(OrcRates)]
            L.orc_tables.argtypes = [dp, dp, dp, dp, C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
            L.orc_threads_available.restype = C.c_int
            L.orc_thermal_q.restype = C.c_int
            L.orc_thermal_q.argtypes = [C.c_void_p]
            L.orc_round_binary16.restype = C.c_double
            L.orc_round_binary16.argtypes = [C.c_double]
            L.orc_set_storage_rounding.argtypes = [C.c_void_p, C.c_int, C.c_double]
            _lib = L
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def tables():
    """The oracle's tables: M (Eq. 13), M^-1 (Eq. A1), N (Eq. 26), N^-1 (Eq. A2),
    the D2Q9 velocities (Eq. 5) and weights (below Eq. 22)."""
    M = np.zeros((9, 9)); Mi = np.zeros((9, 9)); N = np.zeros((5, 5)); Ni = np.zeros((5, 5))
    ex = (C.c_int * 9)(); ey = (C.c_int * 9)(); w = np.zeros(9)
    lib().orc_tables(_dptr(M), _dptr(Mi), _dptr(N), _dptr(Ni), ex, ey, _dptr(w))
    return dict(M=M, Minv=Mi, N=N, Ninv=Ni, ex=np.array(ex[:]), ey=np.array(ey[:]), w=w)


def make_rates(s, z, g_beta=0.0, T0=0.0, ax=0.0, ay=0.0, varpi=0.5, s8_literal=False, theta=1.0,
               bgk=False, rho_in_u=False) -> OrcRates:
    """z has 5 entries (D2Q5 temperature, Eq. 29) or 9 (the D2Q9 model, Eq. 32).
    bgk: single-relaxation-time collisions at omega = s[4], zeta = z[1].
    rho_in_u: the ablation of reading A1 (rho, not rho0, in the velocity-bearing
    terms of the flow collision)."""
    r = OrcRates()
    for k in range(9):
        r.s[k] = float(s[k])
    for k in range(len(z)):
        r.z[k] = float(z[k])
    r.g_beta, r.T0, r.ax, r.ay, r.varpi = g_beta, T0, ax, ay, varpi
    r.s8_literal = int(bool(s8_literal))
    r.tq = 9 if len(z) == 9 else 5
    r.theta = float(theta)
    r.bgk = int(bool(bgk))
    r.rho_in_u = int(bool(rho_in_u))
    return r


def collide_node(rates: OrcRates, fbar, g):
    """One collision (Eq. 8, then Eq. 24 or the D2Q9 model) at one node.
    Returns (f*, g*, (rho, ux, uy, T))."""
    tq = rates.tq
    fbar = np.ascontiguousarray(fbar, dtype=np.float64)
    gin = np.zeros(9)
    gin[:tq] = np.asarray(g, dtype=np.float64)[:tq]
    fo = np.zeros(9); go = np.zeros(9); mac = np.zeros(4)
    lib().orc_collide_node(C.byref(rates), _dptr(fbar), _dptr(gin), _dptr(fo), _dptr(go), _dptr(mac))
    return fo, go[:tq], mac


class OracleLattice:
    """A lattice advanced by the oracle. ``case`` is an ``lbm_cases.Case``.

    Ablations (tests only): ``rho_in_u`` (reading A1), ``s8_literal`` (A2),
    ``nee_uf`` (A11): the fluid node's velocity inside the extrapolated
    non-equilibrium part of node walls, "eq19" (the reading, (j + F/2)/rho0),
    "bare" (j/rho0) or "minus" ((j - F/2)/rho0)."""

    def __init__(self, case, s8_literal: bool = False, threads: int = 1, rho_in_u: bool = False,
                 nee_uf: str = "eq19"):
        self.case = case
        self.nx, self.ny = case.nx, case.ny
        flags = np.ascontiguousarray(case.flags, dtype=np.uint8)
        wu = np.ascontiguousarray([[w.ux, w.uy] for w in case.walls] or [[0.0, 0.0]], dtype=np.float64)
        wk = np.ascontiguousarray([w.kind for w in case.walls] or [0], dtype=np.int32)
        wT = np.ascontiguousarray([w.T for w in case.walls] or [0.0], dtype=np.float64)
        ws = np.ascontiguousarray([getattr(w, "scheme", 0) for w in case.walls] or [0], dtype=np.int32)
        Ti = None if case.T_init is None else np.ascontiguousarray(case.T_init, dtype=np.float64)
        self._keep = (flags, wu, wk, wT, Ti, ws)
        p = OrcParams()
        p.nx, p.ny = case.nx, case.ny
        p.periodic_x, p.periodic_y = int(case.periodic_x), int(case.periodic_y)
        p.flags = flags.ctypes.data
        p.n_walls = len(case.walls)
        p.wall_u, p.wall_kind, p.wall_T = wu.ctypes.data, wk.ctypes.data, wT.ctypes.data
        p.nu, p.alpha, p.g_beta, p.T0 = case.nu, case.alpha, case.g_beta, case.T0
        p.ax, p.ay = case.ax, case.ay
        p.s_e, p.s_q, p.s_eps = case.s_e, case.s_q, case.s_eps
        p.zeta_e, p.zeta_nu, p.varpi = case.zeta_e, case.zeta_nu, case.varpi
        p.s8_literal = int(bool(s8_literal))
        p.T_init = Ti.ctypes.data if Ti is not None else None
        p.wall_scheme = ws.ctypes.data
        p.thermal_q = int(getattr(case, "thermal_q", 5))
        p.theta = float(getattr(case, "theta", 1.0))
        p.zeta_q = float(getattr(case, "zeta_q", 1.0))
        p.zeta_eps = float(getattr(case, "zeta_eps", 1.0))
        p.collision = int(getattr(case, "collision", 0))
        p.rho_in_u_terms = int(bool(rho_in_u))
        # reading A11 (Eq. 19) or an ablation of the fluid node's velocity in the node walls
        p.nee_uf_variant = {"eq19": 0, "bare": 1, "minus": 2}[nee_uf]
        self._p = p
        h = lib().orc_create(C.byref(p))
        if not h:
            raise ValueError("oracle rejected the case (frame, wall ids or size)")
        self._h = h
        if threads != 1:
            lib().orc_set_threads(h, threads)
        self.tq = lib().orc_thermal_q(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def rates(self) -> OrcRates:
        r = OrcRates()
        lib().orc_get_rates(self._h, C.byref(r))
        return r

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def set_storage_rounding(self, bits: int = 16, scale: float = 1.0):
        """Ablation, not the method: after every step, round each population's
        deviation from the rest state (f_bar_i - w_i rho0, g_i - w^T_i T0),
        multiplied by ``scale``, to binary16 (and divide back), as a solver
        storing that deviation in 16 bits would; bits = 0 turns it off. It
        measures the cost of the storage precision alone, the arithmetic
        staying FP64."""
        lib().orc_set_storage_rounding(self._h, int(bits), float(scale))

    def macro(self):
        """(rho, ux, uy, T), each (ny, nx), per reading A6; zeros on solid cells."""
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        lib().orc_macro(self._h, *[_dptr(a) for a in out])
        return tuple(out)

    def populations(self):
        f = np.zeros((9, self.ny, self.nx)); g = np.zeros((self.tq, self.ny, self.nx))
        lib().orc_get_populations(self._h, _dptr(f), _dptr(g))
        return f, g

    def set_populations(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64); g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.size == 9 * self.nx * self.ny and g.size == self.tq * self.nx * self.ny
        lib().orc_set_populations(self._h, _dptr(f), _dptr(g))

    def update_node(self, f_src, g_src, x: int, y: int):
        """One step at node (x, y) reading the external state (f_src, g_src)."""
        fo = np.zeros(9); go = np.zeros(9)
        rc = lib().orc_update_node(self._h, _dptr(f_src), _dptr(g_src), int(x), int(y), _dptr(fo), _dptr(go))
        if rc != 0:
            raise ValueError("solid node")
        return fo, go[:self.tq]

    def nusselt(self, side: int, L: float | None = None, dT: float | None = None) -> float:
        """Mean Nusselt number on a frame wall (Eq. 39, reading A8).
        side: 0 left, 1 right, 2 bottom, 3 top."""
        L = self.case.L if L is None else L
        dT = self.case.delta_T if dT is None else dT
        return lib().orc_nusselt(self._h, int(side), float(L), float(dT))

    def residual(self) -> float:
        """Reading A9 against the previous call's snapshot (+inf on the first call)."""
        return lib().orc_residual(self._h)


def threads_available() -> int:
    return lib().orc_threads_available()


def round_binary16(x: float) -> float:
    """x rounded to the nearest IEEE 754 binary16 value (ties to even),
    returned as a double."""
    return lib().orc_round_binary16(float(x))


def relative_global_error(num, exact) -> float:
    """Relative global error of Eq. 35 (velocity) and Eq. 38 (temperature).

    Eq. 38 is printed as the root of the summed squared deviations over the
    domain divided by the root of the summed squared analytical values; Eq. 35
    names the same L2 norm for the velocity vector. Reading: both are that
    global norm, with the sums over every node and every component of ``num``
    and ``exact`` (arrays of one shape). The alternative reading of Eq. 35 (a
    per-node Euclidean norm summed over the nodes) is kept by the tests for
    comparison."""
    num = np.asarray(num, np.float64)
    exact = np.asarray(exact, np.float64)
    return float(np.sqrt(((num - exact) ** 2).sum() / (exact ** 2).sum()))
