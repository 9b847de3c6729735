"""Many independent problems in one launch (qiht_niht_solve_batched) against the CPU
oracle, problem by problem, and against the single-solve path.

Every problem is quantized with its own seed (codes bit-exact, see
test_gpu_quantize.py); both sides run the same number of iterations. The parity
rule is parity.check: final support, iteration count and reported residual equal while
the oracle's selections are unambiguous, final x within 1e-4 relative L2, otherwise both
recoveries compared with the ground truth."""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_04907_gb300 as q
import parity
import synth

pytestmark = pytest.mark.gpu

def _quantized(problems, bits, base_seed, odd=False):
    out = []
    for i, p in enumerate(problems):
        q1, q2, qy = q.quantize_problem(torch.from_numpy(p.phi).cuda(), torch.from_numpy(p.y).cuda(), bits, bits,
                                        base_seed + i, odd=odd)
        out.append((q1, q2, qy, p.s))
    return out


def _check_against_oracle(res, problems, bits, base_seed, iters, idx, odd=False, label="batch"):
    for i in idx:
        p = problems[i]
        ref, _ = oracle.qiht(p.phi, p.y, p.s, iters, bits_phi=bits, bits_y=bits, seed=base_seed + i, trace=True,
                             odd=odd)
        rep = res.report(i)
        parity.check(f"{label}-{bits}bit[{i}]", ref, p.x_true, x=res.x[i].cpu().numpy(),
                     support=res.support[i].cpu().numpy(), status=rep.status, iters_run=rep.iters_run,
                     resid_norm2=rep.resid_norm2)


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_batch_against_oracle(bits):
    # ragged sizes (m not a multiple of the codes per word, n = 4m); at 2 bits fewer nonzeros
    # per measurement, where the method converges
    s_range = (3, 12) if bits == 2 else (3, 40)
    problems = synth.batch_gaussian(14, seed=40 + bits, m_range=(48, 700), s_range=s_range, snr_db=30.0,
                                    values="pm_u")
    qs = _quantized(problems, bits, 1000)
    res = q.niht_solve_batched(qs, 30)
    torch.cuda.synchronize()
    _check_against_oracle(res, problems, bits, 1000, 30, range(len(problems)))


def test_batch_equals_single_solves():
    # the same problems through qiht_niht_solve one by one: same supports, x within FP32 noise
    problems = synth.batch_gaussian(6, seed=7, m_range=(200, 900), s_range=(5, 30), snr_db=30.0, values="pm_u")
    qs = _quantized(problems, 8, 55)
    res = q.niht_solve_batched(qs, 40)
    singles = [q.niht_solve(q1, q2, qy, s, 40) for (q1, q2, qy, s) in qs]
    torch.cuda.synchronize()
    for i, sv in enumerate(singles):
        rb, rs = res.report(i), sv.read_report()
        assert rb.status == rs.status and rb.iters_run == rs.iters_run, (i, rb, rs)
        assert torch.equal(res.support[i], sv.support), i
        xb, xs = res.x[i].double(), sv.x.double()
        assert float(torch.linalg.norm(xb - xs) / torch.linalg.norm(xs)) < 1e-5, i


def test_batch_shaped_like_the_batched_workload():
    # sizes of the batched workload (m in [128, 2048], n = 4m, s in [8, 128], 4-bit, noiseless),
    # fewer problems; invariants for all, oracle parity for three of them
    problems = synth.batch_gaussian(24, seed=3)
    qs = _quantized(problems, 4, 9000)
    res = q.niht_solve_batched(qs, 25)
    torch.cuda.synchronize()
    reps = res.all_reports()
    for i, p in enumerate(problems):
        assert reps[i].status in (q.OK, q.ERR_BACKTRACK_CAP), (i, reps[i])
        sup = res.support[i].cpu().numpy()
        assert len(np.unique(sup)) == p.s and np.all(np.diff(sup) > 0) and sup.min() >= 0 and sup.max() < p.n
        x = res.x[i].cpu().numpy()
        assert np.all(np.isfinite(x)) and set(np.flatnonzero(x)) <= set(sup)
    sizes = np.array([p.m for p in problems])
    pick = [int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(np.argmax(sizes))]
    _check_against_oracle(res, problems, 4, 9000, 25, pick)


def test_batch_limits_are_checked():
    ok = synth.gaussian(64, 256, 4, seed=1)
    big = synth.gaussian(q.BATCH_MAX_ROWS + 8, 40, 4, seed=2)
    qok = _quantized([ok], 8, 1)[0]
    qbig = _quantized([big], 8, 2)[0]
    with pytest.raises(q.QihtError) as e:
        q.niht_solve_batched([qok, qbig], 5)
    assert e.value.status == q.ERR_ARG
    q4 = _quantized([ok], 4, 3)[0]
    with pytest.raises(q.QihtError) as e:
        q.niht_solve_batched([qok, q4], 5)                 # mixed widths
    assert e.value.status == q.ERR_ARG
    with pytest.raises(q.QihtError) as e:
        q.niht_solve_batched([(qok[0], qok[1], qok[2], q.BATCH_MAX_S + 1)], 5)
    assert e.value.status == q.ERR_ARG


@pytest.mark.parametrize("bits", [2, 8])
def test_batch_odd_grid_against_oracle(bits):
    # every problem on the odd grid of 2^(b-1) + 1 levels, equal-magnitude nonzeros
    s_range = (3, 10) if bits == 2 else (3, 30)
    problems = synth.batch_gaussian(10, seed=60 + bits, m_range=(64, 600), s_range=s_range, snr_db=30.0,
                                    values="ones")
    qs = _quantized(problems, bits, 2000, odd=True)
    res = q.niht_solve_batched(qs, 30)
    torch.cuda.synchronize()
    _check_against_oracle(res, problems, bits, 2000, 30, range(len(problems)), odd=True)


def test_tile_shapes_give_identical_results(monkeypatch):
    # the gradient's tile shape (lanes per column) changes only the order of exact integer sums:
    # every shape the autotuner can pick gives bit-identical solves
    problems = synth.batch_gaussian(12, seed=91, m_range=(64, 2048), s_range=(4, 40), snr_db=30.0, values="pm_u")
    qs = _quantized(problems, 4, 300)
    outs = []
    for shape in ("4", "8", "16", "32"):
        monkeypatch.setenv("QIHT_BATCH_SHAPE", shape)
        res = q.niht_solve_batched(qs, 25)
        torch.cuda.synchronize()
        outs.append(([x.clone() for x in res.x], [r.iters_run for r in res.all_reports()]))
    monkeypatch.delenv("QIHT_BATCH_SHAPE")
    tuned = q.niht_solve_batched(qs, 25)                     # the autotuner's choice
    torch.cuda.synchronize()
    outs.append((tuned.x, [r.iters_run for r in tuned.all_reports()]))
    for xs, its in outs[1:]:
        assert its == outs[0][1]
        assert all(torch.equal(a, b) for a, b in zip(xs, outs[0][0]))
