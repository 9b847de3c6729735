"""The step-size denominator Algorithm 2 prints (QIHT_MU_CROSS) and the residual tolerance, on
the GPU against the oracle, through every iteration path of the library:
  - the persistent iteration kernel for s <= 1024 (graph and eager drivers);
  - the general iteration kernel (s > 1024);
  - the separate-kernel iteration of the fresh-realization solver, where the cross product
    takes the iteration's two new realizations of Q(Phi);
  - the headline size (8192 x 32768, s = 256, 8-bit).
The parity rule is parity.check; with a tolerance, the stopping iteration must be the
oracle's, so the tolerance is placed between two of the oracle's residuals, away from both."""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_04907_gb300 as q
import parity
import synth
from test_gpu_solve import _check, _run_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_cross_step_size_fast_kernel(bits):
    p = synth.gaussian(1000, 3001, 20 if bits > 2 else 8, seed=60 + bits, snr_db=30.0, values="pm_u")
    sv, ref = _run_pair(p, bits, bits, 60, seed=21, mu_mode="cross")
    _check(sv, ref, p, f"cross-{bits}bit")
    # the printed denominator is a different number from the forward square: the runs differ
    fw, _ = oracle.qiht(p.phi, p.y, p.s, 60, bits_phi=bits, bits_y=bits, seed=21, trace=True)
    assert not np.array_equal(fw.trace["mu"], ref.trace["mu"])


def test_cross_step_size_eager_equals_graph():
    p = synth.gaussian(700, 2500, 25, seed=71, snr_db=25.0, values="pm_u")
    phi, y = torch.from_numpy(p.phi).cuda(), torch.from_numpy(p.y).cuda()
    q1, q2, qy = q.quantize_problem(phi, y, 4, 8, 5)
    a = q.niht_solve(q1, q2, qy, p.s, 40, trace=True, mu_mode="cross")
    b = q.niht_solve(q1, q2, qy, p.s, 40, trace=True, mu_mode="cross", eager=True)
    torch.cuda.synchronize()
    assert torch.equal(a.x, b.x) and a.read_report() == b.read_report()
    for k in a.trace:
        assert torch.equal(a.trace[k], b.trace[k]), k


def test_cross_step_size_general_kernel():
    p = synth.gaussian(3000, 6000, 1100, seed=9, snr_db=30.0, values="pm_u")
    sv, ref = _run_pair(p, 8, 8, 20, seed=4, mu_mode="cross")
    _check(sv, ref, p, "cross-s1100")


@pytest.mark.parametrize("bits", [4, 8])
def test_cross_step_size_fresh_realizations(bits):
    # Algorithm 2 as printed: new Phi-hat_{2t-1}, Phi-hat_{2t} in every iteration, and the step
    # size from the product of the two
    p = synth.gaussian(512, 2048, 16, seed=80 + bits, snr_db=30.0, values="pm_u")
    sv = q.niht_solve_fresh(torch.from_numpy(p.phi).cuda(), torch.from_numpy(p.y).cuda(), bits, bits, 5, p.s, 30,
                            trace=True, mu_mode="cross")
    torch.cuda.synchronize()
    ref, _ = oracle.qiht_fresh(p.phi, p.y, p.s, 30, bits_phi=bits, bits_y=bits, seed=5, trace=True, mu_mode="cross")
    _check(sv, ref, p, f"fresh-cross-{bits}bit")


def test_cross_step_size_falls_back_like_the_oracle():
    # at 2 bits with few rows the two quantizations' images of g_G are noisy: some iterations
    # take the forward square; the GPU must take the same branch (supports and mu agree)
    for seed in range(30):
        p = synth.gaussian(40, 160, 6, seed=900 + seed, snr_db=10.0, values="ones")
        ref, _ = oracle.qiht(p.phi, p.y, p.s, 30, bits_phi=2, bits_y=8, seed=seed, trace=True, mu_mode="cross")
        if ref.trace["mu_fallback"].any() and parity.first_ambiguous(ref) is None:
            break
    else:
        pytest.skip("no unambiguous instance with a fallback among the seeds")
    sv, ref = _run_pair(p, 2, 8, 30, seed=seed, mu_mode="cross")
    _check(sv, ref, p, "cross-fallback")


def _tol_between(res, t0):
    r2 = res.trace["resid2"]
    lo, hi = r2[t0], min(r2[1:t0])
    assert lo < 0.85 * hi, "the residual does not drop clearly at t0"
    return float(np.sqrt(lo * hi))          # geometric middle: far from both


@pytest.mark.parametrize("kind", ["fast", "eager", "general", "fresh"])
def test_tolerance_stops_where_the_oracle_stops(kind):
    s = 1100 if kind == "general" else 20
    m, n = (3000, 6000) if kind == "general" else (800, 3000)
    p = synth.gaussian(m, n, s, seed=44, snr_db=30.0, values="pm_u")
    iters = 40
    if kind == "fresh":
        full, _ = oracle.qiht_fresh(p.phi, p.y, s, iters, bits_phi=8, bits_y=8, seed=3, trace=True)
    else:
        full, _ = oracle.qiht(p.phi, p.y, s, iters, bits_phi=8, bits_y=8, seed=3, trace=True)
    t0 = 6 if kind == "general" else 3     # iterations whose residual drops by >= 15 % from the previous ones
    tol = _tol_between(full, t0)
    if kind == "fresh":
        sv = q.niht_solve_fresh(torch.from_numpy(p.phi).cuda(), torch.from_numpy(p.y).cuda(), 8, 8, 3, s, iters,
                                trace=True, tol=tol)
        torch.cuda.synchronize()
        ref, _ = oracle.qiht_fresh(p.phi, p.y, s, iters, bits_phi=8, bits_y=8, seed=3, trace=True, tol=tol)
    else:
        sv, ref = _run_pair(p, 8, 8, iters, seed=3, tol=tol, eager=(kind == "eager"))
    assert ref.iters_run == t0
    rep = sv.read_report()
    assert rep.iters_run == t0 and rep.status == q.OK
    assert rep.resid_norm2 <= tol
    _check(sv, ref, p, f"tol-{kind}")


def test_tolerance_zero_changes_nothing():
    p = synth.gaussian(600, 2000, 15, seed=45, snr_db=30.0, values="pm_u")
    a, _ = _run_pair(p, 4, 4, 25, seed=1)
    b, _ = _run_pair(p, 4, 4, 25, seed=1, tol=0.0)
    assert torch.equal(a.x, b.x) and a.read_report() == b.read_report()


def test_cross_step_size_full_size():
    # the headline configuration with Algorithm 2's printed step size: 8192 x 32768, s = 256,
    # 30 dB, 8-bit, 100 iterations, strict branch required
    p = synth.large_noisy(seed=0)
    sv, ref = _run_pair(p, 8, 8, 100, seed=0, mu_mode="cross")
    _check(sv, ref, p, "large-8bit-cross-100it", require_strict=True)
