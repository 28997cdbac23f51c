"""Mutation tests of the oracle's pins: each case plants one plausible mistake
(a dropped factor, a wrong sign, index or operand, a wrong table entry) in a
copy of oracle/nomrt_oracle.c, compiles it with the oracle's flags, and runs the
CPU pin suites against that build in a subprocess. A pin must fail for every
mutant; a mutant that passes every pin is a hole in the pins.

The mutants cover each part of the method the oracle implements: the moment
tables (Eqs. 13, 26, A1, A2), the weights (below Eq. 22), the velocity (Eq. 19),
the equilibrium moments (Eqs. 16, 28), the forcing (Eq. 17), the collision
(Eqs. 8, 24), the rates (Eqs. 20, 29 and the viscosity/diffusivity relations),
streaming (Eqs. 9, 25), the wall rules (readings A5, A11), the Nusselt
stencils (reading A8), the residual (reading A9), the D2Q9 temperature model
(Eq. 31) and the BGK switch, the buoyancy force (Eq. 4).
"""
import concurrent.futures
import os
import subprocess
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "nomrt_oracle.c")
# every CPU pin of the oracle, in two phases: the quick pins, then the ones
# that run lattices to steady state (a mutant caught by the first phase does
# not wait for the second; -x stops at the first failing pin)
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_d2q9t.py", "tests/test_oracle_bgk.py",
             "tests/test_oracle_nee.py"]
SLOW = "table1 or table2 or slopes or table3 or convergence or onset or stability"
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fopenmp"]

# (name, text in the source, replacement); the text must occur exactly once
MUTANTS = [
    ("M row 7 (Eq. 13)",
     "    {0, 0, 0, 0, 0, 1, -1, -1, 1},\n    {0, 0, 0, 0, 0, 1, 1, 1, 1},\n};",
     "    {0, 0, 0, 0, 0, 1, -1, 1, -1},\n    {0, 0, 0, 0, 0, 1, 1, 1, 1},\n};"),
    ("M^-1 entry (Eq. A1)",
     "{0, 0.5, 0, 0.25, 0.25, 0, 0, -0.5, -0.5},",
     "{0, 0.5, 0, 0.25, -0.25, 0, 0, -0.5, -0.5},"),
    ("N row 4 (Eq. 26)",
     "    {0, 1, -1, 1, -1},\n};",
     "    {0, 1, 1, -1, -1},\n};"),
    ("N^-1 entry (Eq. A2)",
     "    {0, 0, -0.5, 0.25, -0.25},\n};",
     "    {0, 0, -0.5, 0.25, 0.25},\n};"),
    ("diagonal weight",
     "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};",
     "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 9.0};"),
    ("half-force sign in u (Eq. 19)",
     "double uy = (jy + 0.5 * R0 * Fy) / R0;",
     "double uy = (jy - 0.5 * R0 * Fy) / R0;"),
    ("m3_eq density coefficient (Eq. 16)",
     "meq[3] = 2.0 / 3.0 * rho + R0 * uu;",
     "meq[3] = 1.0 / 3.0 * rho + R0 * uu;"),
    ("m8_eq density coefficient (Eq. 16)",
     "meq[8] = 1.0 / 9.0 * rho + 1.0 / 3.0 * R0 * uu;",
     "meq[8] = 1.0 / 3.0 * rho + 1.0 / 3.0 * R0 * uu;"),
    ("m6_eq transposed operand (Eq. 16)",
     "meq[6] = 1.0 / 3.0 * R0 * uy;",
     "meq[6] = 1.0 / 3.0 * R0 * ux;"),
    ("S3 factor (Eq. 17)",
     "S[3] = 2.0 * R0 * (ux * Fx + uy * Fy);",
     "S[3] = R0 * (ux * Fx + uy * Fy);"),
    ("S7 operand (Eq. 17)",
     "S[7] = 1.0 / 3.0 * R0 * Fx;",
     "S[7] = 1.0 / 3.0 * R0 * Fy;"),
    ("forcing weight sign (Eq. 8)",
     "(1.0 - 0.5 * r->s[k]) * S[k];",
     "(1.0 + 0.5 * r->s[k]) * S[k];"),
    ("D2Q5 equilibrium of |c|^2 (Eq. 28)",
     "r->varpi * T, 0.0};",
     "0.5 * r->varpi * T, 0.0};"),
    ("D2Q5 rate per moment (Eq. 24)",
     "for (int k = 0; k < 5; ++k) ns[k] = n[k] - r->z[k] * (n[k] - neq[k]);",
     "for (int k = 0; k < 5; ++k) ns[k] = n[k] - r->z[1] * (n[k] - neq[k]);"),
    ("viscosity relation (Sec. 2.1)",
     "double s_nu = 1.0 / (0.5 + p->nu / CS2);",
     "double s_nu = 1.0 / (0.5 + p->nu * CS2);"),
    ("rates assigned to moments (Eq. 20)",
     "double s[9] = {1.0, 1.0, 1.0, p->s_e, s_nu, s_nu, p->s_q, p->s_q, p->s_eps};",
     "double s[9] = {1.0, 1.0, 1.0, p->s_e, s_nu, s_nu, p->s_eps, p->s_q, p->s_q};"),
    ("D2Q5 diffusivity relation (Sec. 2.2)",
     "double z_alpha = 1.0 / (0.5 + p->alpha / csT2);",
     "double z_alpha = 1.0 / (0.5 + p->alpha / CS2);"),
    ("streaming direction (Eq. 9)",
     "int sx = wrap(x - EX[i], L->nx, L->px);\n",
     "int sx = wrap(x + EX[i], L->nx, L->px);\n"),
    ("moving-wall term factor (A5)",
     "+ 2.0 * W9[i] * RHO0 * (EX[i] * uwx + EY[i] * uwy) / CS2;",
     "+ W9[i] * RHO0 * (EX[i] * uwx + EY[i] * uwy) / CS2;"),
    ("anti-bounce-back constant (A5)",
     "gin[i] = -gsrc[OPP[i] * nxy + self] + 2.0 * even;",
     "gin[i] = -gsrc[OPP[i] * nxy + self] + even;"),
    ("D2Q5 equilibrium advection term (Eq. 30)",
     "return 0.25 * L->r.varpi * T + 0.5 * (EX[i] * ux + EY[i] * uy) * T;",
     "return 0.25 * L->r.varpi * T + 0.25 * (EX[i] * ux + EY[i] * uy) * T;"),
    ("extrapolated non-equilibrium part (A11)",
     "(ff[i] - feq_i(i, rho, ux, uy));",
     "(ff[i] - feq_i(i, rho, uwx, uwy));"),
    ("halfway Nusselt stencil (A8)",
     "(9.0 * T[c1] - T[c2] - 8.0 * Tw) / 3.0;",
     "(9.0 * T[c1] - T[c2] - 8.0 * Tw) / 2.0;"),
    ("node-wall Nusselt stencil (A8, A11)",
     "(-3.0 * Tw + 4.0 * T[c1] - T[c2]) / 2.0",
     "(-3.0 * Tw + 4.0 * T[c1] - T[c2]) / 3.0"),
    ("residual norm (A9)",
     "double Ru = sqrt(num_u) / (du > 1e-300 ? du : 1e-300);",
     "double Ru = num_u / (du > 1e-300 ? du : 1e-300);"),
    ("D2Q9 temperature equilibrium, second-order sign (Eq. 31)",
     "geq[i] = W9[i] * T * (1.0 + eu / CS2 + r->theta * (eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)));",
     "geq[i] = W9[i] * T * (1.0 + eu / CS2 + r->theta * (eu * eu / (2.0 * CS2 * CS2) + uu / (2.0 * CS2)));"),
    ("BGK forcing term sign",
     "(((EX[i] - ux) * Fx + (EY[i] - uy) * Fy) / CS2",
     "(((EX[i] + ux) * Fx + (EY[i] - uy) * Fy) / CS2"),
    ("BGK flow equilibrium, u^2 term",
     "eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2)));\n            double Fi",
     "eu * eu / (2.0 * CS2 * CS2) - uu / CS2));\n            double Fi"),
    ("BGK forcing weight",
     "fstar[i] = fbar[i] - om * (fbar[i] - feq) + (1.0 - 0.5 * om) * Fi;",
     "fstar[i] = fbar[i] - om * (fbar[i] - feq) + (1.0 - om) * Fi;"),
    ("BGK temperature rate",
     "gstar[i] = g[i] - zt * (g[i] - geq);",
     "gstar[i] = g[i] - om * (g[i] - geq);"),
    ("D2Q9 temperature rate per moment (Eq. 32)",
     "for (int k = 0; k < 9; ++k) ns[k] = n[k] - r->z[k] * (n[k] - neq[k]);",
     "for (int k = 0; k < 9; ++k) ns[k] = n[k] - r->z[1] * (n[k] - neq[k]);"),
    ("buoyancy sign (Eq. 4)",
     "double Fy = r->ay + r->g_beta * (T - r->T0);",
     "double Fy = r->ay - r->g_beta * (T - r->T0);"),
    ("buoyancy reference temperature (Eq. 4)",
     "double Fy = r->ay + r->g_beta * (T - r->T0);",
     "double Fy = r->ay + r->g_beta * T;"),
    ("node wall temperature of an adiabatic wall (A11)",
     "double Tb = L->wall_kind[k - 1] == 0 ? L->wall_T[k - 1] : T;",
     "double Tb = L->wall_T[k - 1];"),
    ("nearest fluid node of a boundary node (A11)",
     "for (int i = 1; i < 9 && !d; ++i) {",
     "for (int i = 8; i >= 1 && !d; --i) {"),
    ("residual temperature norm (A9)",
     "double RT = sqrt(num_T) / (dT > 1e-300 ? dT : 1e-300);",
     "double RT = num_T / (dT > 1e-300 ? dT : 1e-300);"),
]


def _source():
    with open(SRC) as f:
        return f.read()


def test_every_mutation_site_exists_once():
    src = _source()
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        assert old != new, name


def _run_mutant(workdir, idx, name, old, new):
    """Compile mutant idx and run the pin suites against it; returns (name,
    exit code, tail of the output). Exit code 1 means a pin failed."""
    src = _source()
    c_path = os.path.join(workdir, f"mutant{idx}.c")
    so_path = os.path.join(workdir, f"libmutant{idx}.so")
    with open(c_path, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", *CFLAGS, c_path, "-o", so_path, "-lm"], check=True)
    env = dict(os.environ, NOMRT_ORACLE_LIB=so_path, OMP_NUM_THREADS="2")
    t0 = time.perf_counter()
    for phase in (f"not ({SLOW})", SLOW):
        r = subprocess.run([sys.executable, "-m", "pytest", *PIN_FILES, "-x", "-q", "-p", "no:cacheprovider",
                            "-m", "not gpu", "-k", phase], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=1200)
        if r.returncode != 0:
            break
    print(f"{name}: exit {r.returncode} after {time.perf_counter() - t0:.1f} s ({phase})")
    return name, r.returncode, r.stdout[-1500:]


def test_pins_catch_every_mutant(tmp_path):
    """Every mutant makes at least one pin fail (the mutants run side by side,
    one process each, on the host's cores)."""
    workers = max(1, min(len(MUTANTS), (os.cpu_count() or 2) // 2))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda a: _run_mutant(str(tmp_path), *a),
                              [(i, *m) for i, m in enumerate(MUTANTS)]))
    # 1: a pin failed; anything else (all passed, or a crash) is not a pin catching it
    survivors = [(name, rc, out) for name, rc, out in results if rc != 1]
    assert not survivors, "mutants that survived the pins:\n" + "\n".join(
        f"{name} (exit {rc}):\n{out}" for name, rc, out in survivors)
