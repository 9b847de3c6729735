import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")
for _p in (ROOT, TESTS):
    if _p not in sys.path:
        sys.path.insert(0, _p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped (not failed) when no GPU is visible, so that
    # `-m gpu` on a CPU machine reports them as skipped.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    # the parity results of this run (tests/parity.py): how many took the strict branch,
    # and the largest errors against the oracle
    try:
        import parity
    except Exception:
        return
    res = parity.RESULTS
    if not res:
        return
    strict = [r for r in res if r.get("branch") == "strict" and "failed" not in r]
    fallback = [r for r in res if r.get("branch") == "fallback" and "failed" not in r]
    failed = [r for r in res if "failed" in r]
    xs = [r["x_rel_vs_oracle"] for r in strict if r.get("x_rel_vs_oracle") is not None]
    r2 = [r.get("resid_norm2_rel") for r in strict if r.get("resid_norm2_rel") is not None]
    line = (f"parity: {len(res)} solve results, {len(strict)} strict, {len(fallback)} fallback, "
            f"{len(failed)} failed")
    if xs:
        line += f"; max x rel vs oracle {max(xs):.2e}"
    if r2:
        line += f"; max ||r||^2 rel {max(r2):.2e}"
    terminalreporter.write_line(line)
    for r in fallback:
        terminalreporter.write_line(f"  fallback: {r['label']} (first ambiguous iteration {r['first_ambiguous']})")
