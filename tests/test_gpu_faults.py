"""Failure detection on the GPU without a fault: a bounded device-side wait that runs out.

The solver's test hook QIHT_SOLVE_TEST_TIMEOUT makes the iteration kernel's CTA 0
withhold its first step-size decision. Every other CTA waits for it with a wait
bounded by the device clock (about 0.2 s); when the bound passes, the kernel records
QIHT_ERR_TIMEOUT in the state and the report and returns. Nothing traps or hangs: the
host reads the status, and the same CUDA context then runs a normal solve.
"""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1802_04907_gb300 as q
import synth

pytestmark = pytest.mark.gpu


def _problem():
    p = synth.gaussian(300, 1000, 10, seed=2, snr_db=30.0)
    phi = torch.from_numpy(p.phi).cuda()
    y = torch.from_numpy(p.y).cuda()
    return p, q.quantize_problem(phi, y, 8, 8, 7)


@pytest.mark.parametrize("eager", [False, True])
def test_forced_timeout_reports_status(eager):
    p, (q1, q2, qy) = _problem()
    sv = q.Solver(p.m, p.n, p.s, 20, eager=eager, test_timeout=True)
    t0 = time.perf_counter()
    sv(q1, q2, qy)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    rep = sv.read_report()
    assert rep.status == q.ERR_TIMEOUT, rep
    assert rep.iters_run == 0
    assert dt < 10.0, dt                         # the waits are bounded (about 0.2 s each)


def test_context_usable_after_timeout():
    p, (q1, q2, qy) = _problem()
    bad = q.Solver(p.m, p.n, p.s, 20, test_timeout=True)
    bad(q1, q2, qy)
    torch.cuda.synchronize()
    assert bad.read_report().status == q.ERR_TIMEOUT
    good = q.Solver(p.m, p.n, p.s, 20)
    good(q1, q2, qy)
    torch.cuda.synchronize()
    rep = good.read_report()
    assert rep.status == q.OK and rep.iters_run == 20
    ref, _ = oracle.qiht(p.phi, p.y, p.s, 20, bits_phi=8, bits_y=8, seed=7)
    assert np.array_equal(np.sort(good.support.cpu().numpy()), ref.support)
