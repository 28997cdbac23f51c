"""The bounds-checking build (-DLBM_BOUNDS), the stand-in for an external
memory checker: tests/bounds_run.py, run with that build loaded, steps tiny
and ragged lattices through every step-kernel variant, storage, model and batch
kind and checks that no access of the step kernels left the lattice's device
block or broke a vector alignment; and that a narrowed range is reported
(without any access outside the block). A subprocess, because a process loads
one build of the library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_no_access_leaves_the_block_in_the_bounds_checking_build():
    env = dict(os.environ, NOMRT_LIB_VARIANT="bounds")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_run.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    print(r.stdout[-2000:], r.stderr[-4000:])
    assert r.returncode == 0, r.stderr[-4000:]
    assert "bounds run ok" in r.stdout
