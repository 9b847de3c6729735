"""The oracle's OpenMP split divides outputs, not sums: every result is bitwise the same for
any number of threads (each column of A^T r, each row of A[:, list] v and each code is
computed by one thread in the serial order)."""
import numpy as np

import oracle
import synth


def _run():
    p = synth.gaussian(300, 1500, 12, seed=8, snr_db=25.0)
    res, q = oracle.qiht(p.phi, p.y, p.s, 25, bits_phi=4, bits_y=8, seed=3, trace=True)
    rng = np.random.Generator(np.random.PCG64(2))
    r = rng.standard_normal(p.m)
    idx = rng.choice(p.n, 40, replace=False).astype(np.int32)
    return (q["codes1"], q["codes2"], oracle.gemv_t(q["A1"], r), oracle.gemv_cols(q["A2"], idx, r[:40]),
            res.x, res.trace["support"], res.trace["mu"], res.trace["resid2"])


def test_results_do_not_depend_on_the_thread_count():
    n0 = oracle.get_threads()
    try:
        oracle.set_threads(1)
        one = _run()
        oracle.set_threads(max(2, n0))
        many = _run()
    finally:
        oracle.set_threads(n0)
    for a, b in zip(one, many):
        assert np.array_equal(a, b)
