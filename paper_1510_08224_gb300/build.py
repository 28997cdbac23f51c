"""Build the in-tree CUDA libraries for sm_103a.

``_build/libnomrt_lbm.so`` is the library; ``_build/libnomrt_lbm_bounds.so``
is the same sources compiled with ``-DLBM_BOUNDS``, the bounds-checking build
whose step kernels test every access against the lattice's device block
(include/nomrt_lbm.h, lbm_bounds_checking). Plain nvcc, one ``-gencode``,
every translation unit of both libraries compiled in parallel and linked with
the CUDA runtime linked statically. No cmake. Rebuilds only what is older
than its sources.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")

# library variant -> (file name, extra nvcc flags)
VARIANTS = {"": ("libnomrt_lbm.so", []), "bounds": ("libnomrt_lbm_bounds.so", ["-DLBM_BOUNDS"])}
LIB = os.path.join(BUILD, VARIANTS[""][0])

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC] + ARCH


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def library_path(variant: str = "") -> str:
    return os.path.join(BUILD, VARIANTS[variant][0])


def is_stale(variant: str = "") -> bool:
    lib = library_path(variant)
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, variants=("", "bounds")) -> str:
    """Compile the stale (or, with force, all) requested variants; returns the
    path of the first one."""
    todo = [v for v in variants if force or is_stale(v)]
    if todo:
        nvcc = _nvcc()
        jobs = []
        for v in todo:
            os.makedirs(os.path.join(BUILD, v or "main"), exist_ok=True)
            jobs += [(v, src) for src in sources()]

        def compile_one(job):
            v, src = job
            obj = os.path.join(BUILD, v or "main", os.path.basename(src)[:-3] + ".o")
            cmd = [nvcc] + NVCC_FLAGS + VARIANTS[v][1] + ["-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src} ({v or 'main'} build):\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                print(r.stdout, r.stderr)
            return v, obj

        workers = max(1, min(16, os.cpu_count() or 1, len(jobs)))
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            done = list(ex.map(compile_one, jobs))
        for v in todo:
            objs = [o for w, o in done if w == v]
            lib = library_path(v)
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc link failed ({v or 'main'} build):\n{r.stdout}\n{r.stderr}")
            os.replace(tmp, lib)
    return library_path(variants[0])


if __name__ == "__main__":
    print(build(force=True, verbose=True))
