"""The parity rule of a GPU solve against the FP64 oracle, shared by the solve tests, and
the record of every result it checks.

Rule (Algorithm 2 run on both sides from bit-identical codes):
  - status equal;
  - strict branch, taken when no iteration of the oracle was ambiguous (relative gap
    between the s-th and (s+1)-th magnitudes of a selection below GAP, or a backtracking
    test within GAP of its threshold): the support after every iteration equal, the
    iteration count equal, the residual ||Q(y) - Q2 x||^2 after every iteration and the
    reported one within RESID_RTOL, the final x within the caller's tolerance (1e-4
    relative L2 for the FP32 paths);
  - up to the first ambiguous iteration otherwise: supports and residuals as above, then
    both recoveries compared against the ground truth (the fallback branch; after an
    ambiguous selection the two trajectories may legitimately differ);
  - step size: where the support changed (mu decides the selection) and in the first three
    iterations, within 1e-4 relative. On every iteration, the displacement of x caused by
    a step-size difference, |mu_gpu - mu_ref| ||g_G||, is at most 1e-4 ||x||: near the
    fixed point g_G vanishes and mu is a ratio of vanishing quantities whose relative
    accuracy degrades like (error of g) / ||g_G||, but its effect on x vanishes with g_G,
    and that effect is what the x tolerance bounds.
Each check appends one JSON record (label, branch, first ambiguous iteration, errors) to
the file named by QIHT_PARITY_LOG (default: .pytest_cache/parity_results.jsonl at the
repository root, a folder git ignores); conftest.py prints a summary at the end of the run.
"""
from __future__ import annotations

import json
import os

import numpy as np

GAP = 1e-5
RESID_RTOL = 1e-4
MU_RTOL = 1e-4
STEP_RTOL = 1e-4

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LOG = os.environ.get("QIHT_PARITY_LOG", os.path.join(_ROOT, ".pytest_cache", "parity_results.jsonl"))
RESULTS: list[dict] = []


def record(rec: dict) -> None:
    RESULTS.append(rec)
    try:
        os.makedirs(os.path.dirname(LOG), exist_ok=True)
        with open(LOG, "a") as f:
            f.write(json.dumps(rec) + "\n")
    except OSError:
        pass


def first_ambiguous(ref, gap: float = GAP) -> int | None:
    tr = ref.trace
    for t in range(ref.iters_run + 1):
        if tr["min_gap"][t] < gap or tr["min_margin"][t] < gap:
            return t
    return None


def _rel(a, b) -> float:
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check(label: str, ref, x_true, **kw) -> dict:
    """Apply the rule to one solve (see _check); a failing check is recorded too."""
    rec = {"label": label}
    try:
        return _check(rec, ref, x_true, **kw)
    except AssertionError as e:
        rec["failed"] = str(e).splitlines()[0][:300]
        record(rec)
        raise


def _check(rec: dict, ref, x_true, *, x, support, status, iters_run, resid_norm2=None, sup_trace=None,
           mu_trace=None, resid_trace=None, x_tol=1e-4, mu_rule="decisive", require_strict=False, gap=GAP,
           resid_rtol=RESID_RTOL) -> dict:
    """Apply the rule to one solve. x, support: the GPU's final iterate and support (numpy);
    *_trace: the GPU's per-iteration records (numpy, rows 0..iters) when it keeps them.
    mu_rule "decisive" checks mu to MU_RTOL where the support changed (and t <= 3) and the
    displacement bound everywhere; "step" checks the displacement bound only.
    A path whose arithmetic is coarser (the FP8 gradient) passes a wider gap, below which the
    oracle's selections count as ambiguous for it, and its own x and residual tolerances.
    Returns the record written."""
    label = rec["label"]
    tr = ref.trace
    amb = first_ambiguous(ref, gap)
    T = ref.iters_run if amb is None else amb - 1
    rec.update({"branch": "strict" if amb is None else "fallback", "first_ambiguous": amb,
                "iters": int(ref.iters_run), "status": int(ref.status)})
    assert status == ref.status, f"{label}: status {status} vs oracle {ref.status}"
    x = np.asarray(x, dtype=np.float64)
    assert np.count_nonzero(x) <= len(ref.support), f"{label}: more than s nonzeros"
    rr2 = tr["resid2"]
    atol = 1e-9 * max(rr2[0], 1e-300)
    if sup_trace is not None:
        for t in range(0, T + 1):
            assert np.array_equal(sup_trace[t], tr["support"][t]), f"{label}: support differs at iteration {t}"
    if resid_trace is not None and T >= 0:
        d = np.abs(resid_trace[: T + 1] - rr2[: T + 1])
        assert np.all(d <= resid_rtol * rr2[: T + 1] + atol), \
            f"{label}: residual differs at iteration {int(np.argmax(d / (rr2[: T + 1] + atol)))}"
        rec["resid2_rel_max"] = float(np.max(d / (rr2[: T + 1] + atol)))
    if mu_trace is not None and T >= 1:
        mu_ref = tr["mu"]
        step = np.abs(mu_trace[1:T + 1] - mu_ref[1:T + 1]) * np.sqrt(tr["num"][1:T + 1])
        lim = STEP_RTOL * np.sqrt(tr["xnorm2"][1:T + 1]) + 1e-30
        assert np.all(step <= lim), f"{label}: step-size displacement at iteration {1 + int(np.argmax(step / lim))}"
        rec["mu_step_rel_max"] = float(np.max(step / np.maximum(np.sqrt(tr["xnorm2"][1:T + 1]), 1e-300)))
        if mu_rule == "decisive":
            worst = 0.0
            for t in range(1, T + 1):
                if t <= 3 or not np.array_equal(tr["support"][t], tr["support"][t - 1]):
                    e = abs(mu_trace[t] - mu_ref[t]) / mu_ref[t]
                    worst = max(worst, e)
                    assert e <= MU_RTOL, f"{label}: mu at {t} differs by {e:.3e}"
            rec["mu_decisive_rel_max"] = worst
    truth = np.linalg.norm(x_true)
    e_gpu = float(np.linalg.norm(x - x_true) / truth) if truth > 0 else None
    e_ref = float(np.linalg.norm(ref.x - x_true) / truth) if truth > 0 else None
    rec.update({"err_gpu_vs_truth": e_gpu, "err_oracle_vs_truth": e_ref})
    if amb is None:
        assert iters_run == ref.iters_run, f"{label}: {iters_run} iterations vs oracle {ref.iters_run}"
        assert np.array_equal(np.sort(np.asarray(support)), ref.support), f"{label}: final support differs"
        rel = _rel(x, ref.x)
        rec["x_rel_vs_oracle"] = rel
        if resid_norm2 is not None:
            rr = abs(resid_norm2 - ref.resid_norm2) / max(ref.resid_norm2, 1e-300)
            rec["resid_norm2_rel"] = float(rr)
            assert abs(resid_norm2 - ref.resid_norm2) <= resid_rtol * ref.resid_norm2 + atol, \
                f"{label}: reported residual {resid_norm2} vs oracle {ref.resid_norm2}"
        assert rel <= x_tol, f"{label}: x differs from the oracle by {rel:.3e}"
        record(rec)
        return rec
    assert not require_strict, f"{label}: the oracle found iteration {amb} ambiguous"
    assert e_gpu <= max(1.5 * e_ref, e_ref + 0.02), f"{label}: gpu error {e_gpu:.3e} vs oracle {e_ref:.3e}"
    record(rec)
    return rec
