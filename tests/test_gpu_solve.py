"""End-to-end parity of qiht_niht_solve (Algorithm 2 on the GPU) with the CPU oracle.

Both sides quantize the same seeded inputs (codes are bit-exact, see
test_gpu_quantize.py) and run the same number of iterations. The GPU computes
g in exact integer sums of 24-bit fixed-point residuals and everything else in
FP32 with FP64 scalars; the oracle is FP64. The rule is parity.check: supports,
residuals and the step size per iteration, then x within 1e-4 relative L2 when no
iteration of the oracle was ambiguous, else both recoveries against the ground truth.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_04907_gb300 as q
import parity
import synth

pytestmark = pytest.mark.gpu

GAP = parity.GAP


def _run_pair(p, bits_phi, bits_y, iters, seed, odd=False, **kw):
    phi = torch.from_numpy(p.phi).cuda()
    y = torch.from_numpy(p.y).cuda()
    q1, q2, qy = q.quantize_problem(phi, y, bits_phi, bits_y, seed, odd=odd)
    sv = q.niht_solve(q1, q2, qy, p.s, iters, trace=True, **kw)
    torch.cuda.synchronize()
    okw = {k: v for k, v in kw.items() if k in ("k", "c", "max_backtrack", "mu_mode", "tol")}
    ref, _ = oracle.qiht(p.phi, p.y, p.s, iters, bits_phi=bits_phi, bits_y=bits_y, seed=seed, trace=True,
                         odd=odd, **okw)
    return sv, ref


def _first_ambiguous(ref):
    return parity.first_ambiguous(ref)


def _check(sv, ref, p, label="", mu_rule="decisive", require_strict=False):
    """parity.check on a Solver's results; returns (x relative to the oracle, None) on the
    strict branch, (None, first ambiguous iteration) on the fallback branch."""
    rep = sv.read_report()
    tr = {k: v.cpu().numpy() for k, v in sv.trace.items()} if sv.trace is not None else {}
    rec = parity.check(label, ref, p.x_true, x=sv.x.cpu().numpy(), support=sv.support.cpu().numpy(),
                       status=rep.status, iters_run=rep.iters_run, resid_norm2=rep.resid_norm2,
                       sup_trace=tr.get("support"), mu_trace=tr.get("mu"), resid_trace=tr.get("resid2"),
                       mu_rule=mu_rule, require_strict=require_strict)
    if rec["branch"] == "strict":
        return rec["x_rel_vs_oracle"], None
    return None, rec["first_ambiguous"]


def test_small_noiseless_8bit():
    # 256 x 1024, s = 16, N(0,1) nonzeros, noiseless, 8-bit Phi and y, 200 iterations, seed 0
    p = synth.small_noiseless(0)
    sv, ref = _run_pair(p, 8, 8, 200, seed=0)
    _check(sv, ref, p, "small")


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_noisy_ragged(bits):
    # sizes not multiples of the tiles: rows 1000 (not a multiple of 16), cols 3001
    p = synth.gaussian(1000, 3001, 25, seed=bits, snr_db=30.0, values="pm_u")
    sv, ref = _run_pair(p, bits, bits, 80, seed=11)
    _check(sv, ref, p, f"ragged-{bits}")


@pytest.mark.parametrize("bits_phi,bits_y", [(2, 8), (4, 8), (8, 4)])
def test_mixed_precision(bits_phi, bits_y):
    p = synth.gaussian(512, 2048, 20, seed=3, snr_db=25.0)
    sv, ref = _run_pair(p, bits_phi, bits_y, 60, seed=5)
    _check(sv, ref, p, f"{bits_phi}/{bits_y}")


@pytest.mark.parametrize("bits", [4, 8])
def test_interferometry_full_size(bits):
    # the interferometry workload at full size: 48 antennas, 2256 baselines, 128 x 128 grid,
    # stacked real 4512 x 16384, 50 sources, 20 dB, s = 64; 20 iterations against the oracle
    p = synth.interferometry(seed=0)
    assert p.phi.shape == (4512, 16384)
    sv, ref = _run_pair(p, bits, bits, 20, seed=2)
    _check(sv, ref, p, f"interferometry-{bits}")


def test_interferometry_small():
    p = synth.interferometry(n_ant=12, grid=32, n_src=6, s=8, snr_db=20.0, seed=2)
    sv, ref = _run_pair(p, 8, 8, 60, seed=1)
    _check(sv, ref, p, "interferometry")


def test_mri_small():
    # MRI-shaped: radial k-space samples (a third of a 32 x 32 grid) of a Haar-sparse head image,
    # stacked real 696 x 1024, s = 48, 30 dB, 8-bit
    p = synth.mri(grid=32, s=48, seed=1)
    sv, ref = _run_pair(p, 8, 8, 100, seed=3)
    # on this operator the iteration amplifies rounding in mu (it drifts from the FP64
    # iteration by more than 1e-4 relative after a few tens of iterations while x stays
    # within ~1e-6): mu is held to the displacement bound on every iteration, supports,
    # residuals and x as everywhere
    _check(sv, ref, p, "mri-32", mu_rule="step")


def test_mri_full_size():
    # the MRI-shaped workload at full size: 128 x 128 image, stacked real 11364 x 16384, s = 512,
    # 30 dB, 8-bit; 20 iterations against the oracle
    p = synth.mri(seed=0)
    assert p.phi.shape == (11364, 16384)
    sv, ref = _run_pair(p, 8, 8, 20, seed=2)
    _check(sv, ref, p, "mri-128")


def test_backtracking_instance():
    # equal magnitudes, low SNR: shrinks happen; their count must match where unambiguous
    for seed in range(40):
        p = synth.gaussian(48, 128, 12, seed=300 + seed, values="ones", snr_db=10.0)
        ref, _ = oracle.qiht(p.phi, p.y, 12, 40, bits_phi=8, bits_y=8, seed=seed, trace=True)
        if ref.backtracks > 0:
            break
    sv, ref = _run_pair(p, 8, 8, 40, seed=seed)
    _check(sv, ref, p, "backtracking")
    amb = parity.first_ambiguous(ref)
    T = ref.iters_run if amb is None else amb - 1
    bt = sv.trace["bt"].cpu().numpy()
    assert np.array_equal(bt[1:T + 1], ref.trace["bt"][1:T + 1])


def test_zero_iterations_gives_initial_support():
    p = synth.gaussian(200, 700, 9, seed=4)
    sv, ref = _run_pair(p, 8, 8, 0, seed=2)
    rep = sv.read_report()
    assert rep.iters_run == 0 and rep.status == q.OK
    assert torch.all(sv.x == 0)
    assert np.array_equal(sv.support.cpu().numpy(), ref.support)


def test_zero_observation_converges_immediately():
    p = synth.gaussian(64, 256, 4, seed=1)
    p.y[:] = 0.0
    sv, ref = _run_pair(p, 8, 8, 10, seed=1)
    rep = sv.read_report()
    assert rep.iters_run == 0 == ref.iters_run and rep.status == q.OK
    assert torch.all(sv.x == 0)


def test_nonfinite_input_reports_status():
    p = synth.gaussian(64, 256, 4, seed=1)
    p.phi[3, 3] = np.nan
    phi = torch.from_numpy(p.phi).cuda()
    y = torch.from_numpy(p.y).cuda()
    q1, q2, qy = q.quantize_problem(phi, y, 8, 8, 1)
    sv = q.niht_solve(q1, q2, qy, 4, 10)
    torch.cuda.synchronize()
    assert sv.read_report().status == q.ERR_NONFINITE


def test_deterministic_and_graph_reuse():
    p = synth.gaussian(700, 2500, 30, seed=8, snr_db=20.0)
    phi = torch.from_numpy(p.phi).cuda()
    y = torch.from_numpy(p.y).cuda()
    q1, q2, qy = q.quantize_problem(phi, y, 4, 4, 3)
    sv = q.Solver(700, 2500, 30, 50)
    sv(q1, q2, qy)
    torch.cuda.synchronize()
    x1 = sv.x.clone()
    r1 = sv.read_report()
    sv(q1, q2, qy)          # same pointers: cached graph
    torch.cuda.synchronize()
    assert torch.equal(sv.x, x1)
    assert sv.read_report() == r1


@pytest.mark.parametrize("bits,iters", [(8, 300), (4, 60)])
def test_full_size_large_solve_against_oracle(bits, iters):
    # the benchmarked configuration at full size: 8192 x 32768, s = 256, +-U(0.5,1.5)
    # nonzeros, 30 dB; 8-bit with the full 300 iterations, 4-bit with 60. The oracle solves
    # the same quantized instance in FP64 (two 2 GiB matrices); no iteration of it is
    # ambiguous, so the strict branch is required: supports and residuals at every
    # iteration, the step sizes, and x within 1e-4 of the oracle's
    p = synth.large_noisy(seed=0)
    sv, ref = _run_pair(p, bits, bits, iters, seed=0)
    rel, amb = _check(sv, ref, p, f"large-{bits}bit-{iters}it", require_strict=True)
    assert amb is None
    rep = sv.read_report()
    assert rep.status == q.OK
    x = sv.x.cpu().numpy().astype(np.float64)
    assert set(np.flatnonzero(x)) <= set(sv.support.cpu().numpy())
    if bits == 8:
        assert len(np.intersect1d(sv.support.cpu().numpy(), p.support)) >= 0.99 * p.s
        assert np.linalg.norm(x - p.x_true) / np.linalg.norm(p.x_true) < 0.05


def test_eager_driver_matches_graph():
    # the host-driven launch sequence runs the same kernels as the graph: identical results
    for seed in range(20):
        p = synth.gaussian(300, 1200, 24, seed=500 + seed, values="ones", snr_db=8.0)
        ref, _ = oracle.qiht(p.phi, p.y, p.s, 30, bits_phi=4, bits_y=8, seed=seed)
        if ref.backtracks > 0:
            break
    phi = torch.from_numpy(p.phi).cuda()
    y = torch.from_numpy(p.y).cuda()
    q1, q2, qy = q.quantize_problem(phi, y, 4, 8, seed)
    a = q.Solver(p.m, p.n, p.s, 30, trace=True)
    b = q.Solver(p.m, p.n, p.s, 30, trace=True, eager=True)
    a(q1, q2, qy)
    b(q1, q2, qy)
    torch.cuda.synchronize()
    assert torch.equal(a.x, b.x) and torch.equal(a.support, b.support)
    assert a.read_report() == b.read_report()
    for k in a.trace:
        assert torch.equal(a.trace[k], b.trace[k]), k


def test_large_support_uses_the_general_iteration_kernel():
    # s above the shared-memory lists of the fast iteration kernel (1024): the general kernel
    # (filter and one-CTA select inside the kernel) runs every iteration
    p = synth.gaussian(3000, 6000, 1100, seed=9, snr_db=30.0, values="pm_u")
    sv, ref = _run_pair(p, 8, 8, 25, seed=4)
    _check(sv, ref, p, "s=1100")


def test_fast_and_general_iteration_kernels_agree(tmp_path):
    # the same solve through both iteration kernels (QIHT_ITER=base selects the general one;
    # it is read once per process, hence the subprocess)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "solve.py"
    script.write_text(
        "import sys, numpy as np, torch\n"
        f"sys.path.insert(0, {root!r})\n"
        "import paper_1802_04907_gb300 as q, synth\n"
        "p = synth.gaussian(900, 3000, 30, seed=21, snr_db=25.0, values='pm_u')\n"
        "phi = torch.from_numpy(p.phi).cuda(); y = torch.from_numpy(p.y).cuda()\n"
        "q1, q2, qy = q.quantize_problem(phi, y, 8, 8, 6)\n"
        "sv = q.niht_solve(q1, q2, qy, p.s, 60, trace=True)\n"
        "torch.cuda.synchronize()\n"
        "r = sv.read_report()\n"
        "np.savez(sys.argv[1], x=sv.x.cpu().numpy(), sup=sv.trace['support'].cpu().numpy(),\n"
        "         iters=r.iters_run, status=r.status)\n")
    outs = {}
    for kind in ("base", "fast"):
        env = dict(os.environ)
        if kind == "base":
            env["QIHT_ITER"] = "base"
        else:
            env.pop("QIHT_ITER", None)
        out = tmp_path / f"{kind}.npz"
        subprocess.run([sys.executable, str(script), str(out)], env=env, check=True, timeout=300)
        outs[kind] = np.load(out)
    a, b = outs["base"], outs["fast"]
    assert int(a["status"]) == int(b["status"]) == q.OK
    assert int(a["iters"]) == int(b["iters"])
    assert np.array_equal(a["sup"], b["sup"])
    rel = np.linalg.norm(a["x"] - b["x"]) / np.linalg.norm(a["x"])
    assert rel < 1e-5, rel


@pytest.mark.parametrize("env", [{"QIHT_PDL": "0"}, {"QIHT_UNROLL": "1"}, {"QIHT_UNROLL": "3"},
                                 {"QIHT_PDL": "0", "QIHT_UNROLL": "5"}])
def test_graph_variants_match_the_default_graph(tmp_path, env):
    # the solver graph built without programmatic edges, or with another number of iterations
    # per loop-body execution, runs the same kernels on the same data: bitwise equal results
    # (both switches are read once per process, hence the subprocesses)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "solve.py"
    script.write_text(
        "import sys, numpy as np, torch\n"
        f"sys.path.insert(0, {root!r})\n"
        "import paper_1802_04907_gb300 as q, synth\n"
        "p = synth.gaussian(900, 3000, 30, seed=21, snr_db=25.0, values='pm_u')\n"
        "phi = torch.from_numpy(p.phi).cuda(); y = torch.from_numpy(p.y).cuda()\n"
        "q1, q2, qy = q.quantize_problem(phi, y, 4, 8, 6)\n"
        "sv = q.niht_solve(q1, q2, qy, p.s, 37, trace=True)\n"
        "torch.cuda.synchronize()\n"
        "r = sv.read_report()\n"
        "np.savez(sys.argv[1], x=sv.x.cpu().numpy(), sup=sv.trace['support'].cpu().numpy(),\n"
        "         mu=sv.trace['mu'].cpu().numpy(), r2=sv.trace['resid2'].cpu().numpy(),\n"
        "         rep=np.array([r.iters_run, r.status, r.backtracks, r.support_changes]), rn=r.resid_norm2)\n")
    outs = {}
    for kind, extra in (("default", {}), ("variant", env)):
        e = {k: v for k, v in os.environ.items() if k not in ("QIHT_PDL", "QIHT_UNROLL")}
        e.update(extra)
        out = tmp_path / f"{kind}.npz"
        subprocess.run([sys.executable, str(script), str(out)], env=e, check=True, timeout=300)
        outs[kind] = np.load(out)
    a, b = outs["default"], outs["variant"]
    assert int(a["rep"][0]) == 37 and int(a["rep"][1]) == q.OK
    for k in ("x", "sup", "mu", "r2", "rep", "rn"):
        assert np.array_equal(a[k], b[k]), k


def test_exact_ties_resolve_by_index():
    # +-1 entries quantize deterministically (they sit on the two end levels), so duplicated
    # columns have identical codes and identical gradients: H_s must break the ties by the
    # lower index, on both sides, in every iteration
    dup = 4
    p = synth.duplicated_pm1(64, 96, dup, 5, seed=17)
    sv, ref = _run_pair(p, 8, 8, 30, seed=3)
    rep = sv.read_report()
    assert rep.status == ref.status == q.OK
    assert rep.iters_run == ref.iters_run
    sup = sv.trace["support"].cpu().numpy()
    for t in range(ref.iters_run + 1):
        assert np.array_equal(sup[t], ref.trace["support"][t]), f"support differs at iteration {t}"
    xg = sv.x.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x)
    assert rel < 1e-4, rel


# ---- the odd grid (2^(b-1) + 1 levels with a zero level, the Appendix's remark) ----

@pytest.mark.parametrize("bits", [2, 4, 8])
def test_odd_grid_noisy_ragged(bits):
    p = synth.gaussian(1000, 3001, 25, seed=10 + bits, snr_db=30.0, values="pm_u")
    sv, ref = _run_pair(p, bits, bits, 80, seed=13, odd=True)
    _check(sv, ref, p, f"odd-ragged-{bits}")


@pytest.mark.parametrize("bits_phi,bits_y", [(2, 8), (4, 4)])
def test_odd_grid_equal_magnitudes(bits_phi, bits_y):
    # nonzeros of x all equal to 1 (the paper's harder synthetic case), mixed widths
    p = synth.gaussian(512, 2048, 20, seed=7, snr_db=25.0, values="ones")
    sv, ref = _run_pair(p, bits_phi, bits_y, 60, seed=4, odd=True)
    _check(sv, ref, p, f"odd-ones-{bits_phi}/{bits_y}")


def test_odd_grid_interferometry_full_size():
    # the interferometry workload at full size (stacked real 4512 x 16384, s = 64) on the 8-bit
    # odd grid (129 levels): 20 iterations against the oracle
    p = synth.interferometry(seed=0)
    sv, ref = _run_pair(p, 8, 8, 20, seed=3, odd=True)
    _check(sv, ref, p, "odd-interferometry")
