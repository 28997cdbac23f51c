import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test (tens of seconds)")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """One line per test file with its passed / failed / skipped counts, so a
    quiet run's log still records which files ran (the no-alloc entry point's
    file among them)."""
    per = {}
    for kind in ("passed", "failed", "skipped", "error"):
        for rep in terminalreporter.stats.get(kind, []):
            nodeid = getattr(rep, "nodeid", "")
            if not nodeid or getattr(rep, "when", "call") not in ("call", "setup"):
                continue
            if kind == "passed" and rep.when != "call":
                continue
            f = nodeid.split("::")[0]
            per.setdefault(f, {}).setdefault(kind, 0)
            per[f][kind] += 1
    if not per:
        return
    terminalreporter.write_line("per-file results:")
    for f in sorted(per):
        counts = ", ".join(f"{n} {k}" for k, n in sorted(per[f].items()))
        terminalreporter.write_line(f"  {f}: {counts}")
