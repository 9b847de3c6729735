"""Writes the stored expected values in this directory by calling only the CPU oracle.

    python tests/golden/make_golden.py

The fixtures freeze the oracle's results on small seeded inputs: quantization codes on both
grids (Section III-A; the odd grid of the Appendix's remark), a short solve of Algorithm 2 with
its per-iteration supports, a run with fresh realizations per iteration, and the gradients of
the unrolled iterations. tests/test_golden.py checks that the oracle still reproduces them (a
change of its arithmetic must say which passage of the paper justifies it). No value here comes
from the CUDA library."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import unrolled  # noqa: E402
import synth  # noqa: E402


def main():
    v = synth.random_floats((9, 7), seed=1)
    codes = {}
    for bits in (2, 4, 8):
        for odd in (False, True):
            c, sc = oracle.quantize(v, bits, seed=12345, stream=3, odd=odd)
            codes[f"b{bits}{'_odd' if odd else ''}"] = {"codes": c.tolist(), "scale": sc}
    p = synth.gaussian(48, 160, 5, seed=7, snr_db=30.0, values="pm_u")
    res, _ = oracle.qiht(p.phi, p.y, p.s, 12, bits_phi=4, bits_y=8, seed=11, trace=True)
    fr, _ = oracle.qiht_fresh(p.phi, p.y, p.s, 6, bits_phi=8, bits_y=8, seed=11, trace=True)
    c1, sc = oracle.quantize(p.phi, 4, 5, 0)
    c2, _ = oracle.quantize(p.phi, 4, 5, 1, sc)
    P1, P2 = oracle.dequantize(c1, 4, sc), oracle.dequantize(c2, 4, sc)
    m = p.phi.shape[0]
    rng = np.random.Generator(np.random.PCG64(3))
    a, b = rng.uniform(0.9, 1.1, m), rng.uniform(-0.1, 0.1, m)
    yy = np.concatenate([a * p.y, b * p.y])
    L, gy, ga, gb, _, _ = unrolled.loss_and_grads(P1, P2, yy, a, b, p.s, 4, p.x_true)
    out = {
        "quantize": {"input_seed": 1, "shape": [9, 7], "seed": 12345, "stream": 3, "grids": codes},
        "solve": {"problem": "synth.gaussian(48, 160, 5, seed=7, snr_db=30.0, values='pm_u')",
                  "bits_phi": 4, "bits_y": 8, "seed": 11, "iters": 12,
                  "supports": res.trace["support"].tolist(), "x": res.x.tolist(),
                  "resid_norm2": res.resid_norm2, "backtracks": res.backtracks},
        "fresh": {"bits": 8, "seed": 11, "iters": 6, "supports": fr.trace["support"].tolist(), "x": fr.x.tolist()},
        "unrolled": {"bits": 4, "seed": 5, "K": 4, "gain_seed": 3, "loss": L, "gy": gy.tolist(),
                     "ga": ga.tolist(), "gb": gb.tolist()},
    }
    with open(os.path.join(HERE, "oracle_results.json"), "w") as f:
        json.dump(out, f)
        f.write("\n")


if __name__ == "__main__":
    main()
