"""The oracle reproduces the stored results in tests/golden/oracle_results.json (written by
tests/golden/make_golden.py from the oracle alone): quantization codes on both grids, a solve
of Algorithm 2 with its supports, a run with fresh realizations, unrolled gradients. Codes and
supports must match exactly, floating-point results to 1e-12 relative."""
import json
import os

import numpy as np

import oracle
from oracle import unrolled
import synth

G = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_results.json")))


def test_quantization_codes():
    q = G["quantize"]
    v = synth.random_floats(tuple(q["shape"]), seed=q["input_seed"])
    for name, rec in q["grids"].items():
        bits = int(name[1])
        c, sc = oracle.quantize(v, bits, seed=q["seed"], stream=q["stream"], odd=name.endswith("odd"))
        assert np.array_equal(c, np.array(rec["codes"])), name
        assert sc == rec["scale"]


def test_solve_supports_and_result():
    r = G["solve"]
    p = synth.gaussian(48, 160, 5, seed=7, snr_db=30.0, values="pm_u")
    res, _ = oracle.qiht(p.phi, p.y, p.s, r["iters"], bits_phi=r["bits_phi"], bits_y=r["bits_y"], seed=r["seed"],
                         trace=True)
    assert np.array_equal(res.trace["support"], np.array(r["supports"]))
    assert np.allclose(res.x, r["x"], rtol=1e-12, atol=0)
    assert abs(res.resid_norm2 - r["resid_norm2"]) <= 1e-12 * r["resid_norm2"]
    assert res.backtracks == r["backtracks"]


def test_fresh_and_unrolled():
    p = synth.gaussian(48, 160, 5, seed=7, snr_db=30.0, values="pm_u")
    f = G["fresh"]
    fr, _ = oracle.qiht_fresh(p.phi, p.y, p.s, f["iters"], bits_phi=f["bits"], bits_y=f["bits"], seed=f["seed"],
                              trace=True)
    assert np.array_equal(fr.trace["support"], np.array(f["supports"]))
    assert np.allclose(fr.x, f["x"], rtol=1e-12, atol=0)
    u = G["unrolled"]
    c1, sc = oracle.quantize(p.phi, u["bits"], u["seed"], 0)
    c2, _ = oracle.quantize(p.phi, u["bits"], u["seed"], 1, sc)
    P1, P2 = oracle.dequantize(c1, u["bits"], sc), oracle.dequantize(c2, u["bits"], sc)
    m = p.phi.shape[0]
    rng = np.random.Generator(np.random.PCG64(u["gain_seed"]))
    a, b = rng.uniform(0.9, 1.1, m), rng.uniform(-0.1, 0.1, m)
    yy = np.concatenate([a * p.y, b * p.y])
    L, gy, ga, gb, _, _ = unrolled.loss_and_grads(P1, P2, yy, a, b, p.s, u["K"], p.x_true)
    assert abs(L - u["loss"]) <= 1e-12 * abs(u["loss"])
    for got, key in ((gy, "gy"), (ga, "ga"), (gb, "gb")):
        assert np.allclose(got, u[key], rtol=1e-10, atol=1e-14)
