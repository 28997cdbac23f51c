"""Runs in a subprocess with NOMRT_LIB_VARIANT=bounds (see test_gpu_bounds.py):
the bounds-checking build of the library, whose step kernels test every
population, link-map, flag and wall-table access against the lattice's device
block before making it and record the first refusal.

1. Tiny and ragged lattices (widths 1, 5, 6, 7, 133, 261; periodic in x, in
   y, in both; halfway and node-based walls; scattered solid cells), in every
   storage, with every step-kernel variant and config, with the D2Q5 and D2Q9
   temperature models and the MRT and BGK collisions, and batched in every
   batch kind (the fused kind also with one row segment per warp): after 3 steps from an off-equilibrium state no access was
   refused (the synchronising read-out would raise), and the FP64 result still
   equals the oracle's.
2. The detector: a lattice whose checks accept only the first half of its
   block reports a refused access (LBM_ECUDA naming a site) at the next
   synchronising call, and runs clean again once the full block is restored.
   No access outside the block is made in either case.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import lbm_cases as lc  # noqa: E402
import oracle  # noqa: E402


def cases():
    return [
        lc.periodic_box(7, 5, nu=0.03, alpha=0.04, g_beta=2e-3, T0=0.5,
                        kinetic=dict(s_e=1.3, s_q=1.1, s_eps=1.5, zeta_e=1.2, zeta_nu=0.9), ax=1e-5),
        lc.periodic_box(1, 1, nu=0.03, alpha=0.04),
        lc.couette(H=9, nx=5, U0=0.05),
        lc.cavity(n=20, Ra=1e4, n_y=13, noise=1e-3),
        lc.rayleigh_benard(nx=133, H=7, Ra=1e5, sigma=1e-2),
        lc.poiseuille(H=11, nx=1, ax=1e-5),
        lc.obstacle_channel(nx=261, H=9, frac=0.15, seed=4),
        lc.periodic_box(6, 9, nu=0.02, alpha=0.03, T0=0.2, T_init=0.2 + 0.1 * lc.uniform01(9, 54).reshape(9, 6)),
        lc.cavity_nee(n=19, Ra=1e4, noise=1e-3),
        lc.porous_couette_nee(H=13, nx=5, Re=10, s_nu=0.8),
    ]


def main():
    import torch
    import paper_1510_08224_gb300 as P
    L = P.load()
    assert P.library_path().endswith("libnomrt_lbm_bounds.so"), P.library_path()
    assert L.lbm_bounds_checking() == 1, "not the bounds-checking build"
    torch.cuda.set_device(0)
    runs = 0
    for i, base in enumerate(cases()):
        models = [base, lc.with_bgk(base)]
        if base.name not in ("cavity_nee", "porous_couette_nee"):
            models.append(lc.with_d2q9_temperature(base))
        for case in models:
            f0, g0 = lc.random_state(case, seed=90 + i)
            for st in ("f64", "f32", "f16"):
                for v in [("auto", 0)] + P.step_kernels(st):
                    lat = P.Lattice(case, storage=st)
                    try:
                        lat.set_step_kernel(*v)
                    except P.LBMError:
                        lat.close()
                        continue  # this model has no such variant
                    lat.set_populations(f0, g0)
                    lat.step(3)
                    lat.sync()
                    mac = lat.macro()  # synchronises: raises if an access was refused
                    if st == "f64" and v == ("auto", 0):
                        o = oracle.OracleLattice(case)
                        o.set_populations(f0, g0)
                        o.step(3)
                        for a, b in zip(mac, o.macro()):
                            assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max()), (case.name, st)
                    lat.close()
                    runs += 1
    # batches: every kind, members of uneven size with both wall schemes
    mix = [c for c in cases() if c.nx * c.ny > 1]
    halfway = [c for c in mix if not c.name.endswith("nee")]
    for st in ("f32", "f16"):
        for kind, members, cfg in (("fused", mix, -1), ("fused", mix, 6), ("persistent", halfway, -1),
                                   ("concurrent", mix, -1)):
            b = P.Batch()
            b.set_kind(kind)
            b.set_mode(3, 0)
            b.set_config(cfg, 1)
            lats = []
            for i, c in enumerate(members):
                lat = P.Lattice(c, storage=st)
                f0, g0 = lc.random_state(c, seed=120 + i)
                lat.set_populations(f0, g0)
                b.add(lat)
                lats.append(lat)
            b.step(7)
            b.sync()  # raises if a member's access was refused
            for lat in lats:
                lat.macro()
            b.close()
            runs += 1
    # the detector fires on a narrowed range and clears again
    case = lc.cavity(n=40, Ra=1e4, noise=1e-3)
    lat = P.Lattice(case, storage="f32")
    h = lat.handle
    assert L.lbm_debug_bounds_limit(h, lat.footprint // 2) == 0
    lat.step(2)
    try:
        lat.sync()
        raise AssertionError("a narrowed range must be reported")
    except P.LBMError as e:
        assert e.status == 3 and "site" in str(e), e
    assert L.lbm_debug_bounds_limit(h, lat.footprint) == 0
    lat.set_populations(*lc.random_state(case, seed=5))
    lat.step(2)
    lat.sync()
    lat.macro()
    lat.close()
    print(f"bounds run ok: {runs} runs, no access refused; a narrowed range is reported", flush=True)


if __name__ == "__main__":
    main()
