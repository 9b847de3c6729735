"""Algorithm 2 with fresh realizations per iteration (qiht_niht_solve_fresh) against the
CPU oracle's qiht_fresh on the same seeded inputs; the parity rule is the one of
test_gpu_solve.py (supports identical at every iteration while the oracle's selections are
unambiguous, step sizes within 1e-4, final x within 1e-4 relative L2, otherwise both
recoveries compared with the ground truth). Also: iteration 1 equals the fixed-quantization
solve, and the fixed solve through the separate-kernel iteration path agrees with the
default path."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import paper_1802_04907_gb300 as q
import synth
from test_gpu_solve import _check

pytestmark = pytest.mark.gpu


def _fresh_pair(p, bits_phi, bits_y, iters, seed, odd=False):
    sv = q.niht_solve_fresh(torch.from_numpy(p.phi).cuda(), torch.from_numpy(p.y).cuda(), bits_phi, bits_y, seed,
                            p.s, iters, odd=odd, trace=True)
    torch.cuda.synchronize()
    ref, _ = oracle.qiht_fresh(p.phi, p.y, p.s, iters, bits_phi=bits_phi, bits_y=bits_y, seed=seed, trace=True,
                               odd=odd)
    return sv, ref


@pytest.mark.parametrize("bits", [4, 8])
def test_fresh_against_oracle(bits):
    p = synth.gaussian(512, 2048, 16, seed=30 + bits, snr_db=30.0, values="pm_u")
    sv, ref = _fresh_pair(p, bits, bits, 30, seed=5)
    _check(sv, ref, p, f"fresh-{bits}")


def test_fresh_ragged_mixed_widths():
    # rows not a multiple of the codes per word, columns off every tile; 4-bit Phi, 8-bit y
    p = synth.gaussian(1000, 3001, 12, seed=8, snr_db=30.0, values="pm_u")
    sv, ref = _fresh_pair(p, 4, 8, 25, seed=2)
    _check(sv, ref, p, "fresh-ragged")


def test_fresh_odd_grid():
    p = synth.gaussian(384, 1536, 12, seed=14, snr_db=30.0, values="ones")
    sv, ref = _fresh_pair(p, 8, 8, 25, seed=11, odd=True)
    _check(sv, ref, p, "fresh-odd")


def test_fresh_first_iteration_equals_fixed_solve():
    p = synth.gaussian(700, 2800, 20, seed=3, snr_db=30.0, values="pm_u")
    phi, y = torch.from_numpy(p.phi).cuda(), torch.from_numpy(p.y).cuda()
    fr = q.niht_solve_fresh(phi, y, 8, 8, 9, p.s, 1)
    q1, q2, qy = q.quantize_problem(phi, y, 8, 8, 9)
    fx = q.niht_solve(q1, q2, qy, p.s, 1)
    torch.cuda.synchronize()
    assert torch.equal(torch.sort(fr.support).values, torch.sort(fx.support).values)
    rel = (torch.linalg.norm(fr.x - fx.x) / torch.linalg.norm(fx.x)).item()
    assert rel < 1e-5, rel


def test_separate_kernel_iteration_path_agrees(tmp_path):
    # the fixed solve with the iteration as separate kernels (QIHT_SOLVER=multi, read once per
    # process) against the default persistent iteration kernel
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "solve.py"
    script.write_text(
        "import sys, numpy as np, torch\n"
        f"sys.path.insert(0, {root!r})\n"
        "import paper_1802_04907_gb300 as q, synth\n"
        "p = synth.gaussian(900, 3000, 30, seed=22, snr_db=25.0, values='pm_u')\n"
        "phi = torch.from_numpy(p.phi).cuda(); y = torch.from_numpy(p.y).cuda()\n"
        "q1, q2, qy = q.quantize_problem(phi, y, 8, 8, 6)\n"
        "sv = q.niht_solve(q1, q2, qy, p.s, 60, trace=True)\n"
        "torch.cuda.synchronize()\n"
        "r = sv.read_report()\n"
        "np.savez(sys.argv[1], x=sv.x.cpu().numpy(), sup=sv.trace['support'].cpu().numpy(),\n"
        "         iters=r.iters_run, status=r.status)\n")
    outs = {}
    for kind in ("multi", "default"):
        env = dict(os.environ)
        if kind == "multi":
            env["QIHT_SOLVER"] = "multi"
        else:
            env.pop("QIHT_SOLVER", None)
        out = tmp_path / f"{kind}.npz"
        subprocess.run([sys.executable, str(script), str(out)], env=env, check=True, timeout=300)
        outs[kind] = np.load(out)
    a, b = outs["multi"], outs["default"]
    assert int(a["status"]) == int(b["status"]) == q.OK
    assert int(a["iters"]) == int(b["iters"])
    assert np.array_equal(a["sup"], b["sup"])
    assert np.linalg.norm(a["x"] - b["x"]) / np.linalg.norm(a["x"]) < 1e-5
