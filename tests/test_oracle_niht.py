"""Pins for the oracle's normalized IHT / QIHT (Algorithms 1 and 2).

Checks fixed by mathematics or by the paper, independent of the oracle:
  - brute force: on tiny instances (n <= 16) every support is enumerated and
    solved by least squares; NIHT must reach the global optimum on noiseless
    instances
  - exact recovery of a noiseless s-sparse signal from a Gaussian matrix
  - ||x||_0 <= s after every step; H_s equals a stable library sort
  - the adaptive step lies in [1/sigma_max^2, 1/sigma_min^2] of Phi_Gamma
    (Section II-A: it is a Rayleigh quotient)
  - the backtracking condition mu <= (1-c) omega holds whenever the support changes
  - with Q1 = Q2 the cost ||y - Phi x||^2 never increases (Section III-B, Theorem 3)
  - double sampling gives an unbiased gradient (Section III-A)
  - QIHT with many bits approaches NIHT
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


def _brute_force(phi, y, s):
    best = (np.inf, None, None)
    n = phi.shape[1]
    for sup in itertools.combinations(range(n), s):
        A = phi[:, sup]
        coef, *_ = np.linalg.lstsq(A, y, rcond=None)
        cost = float(np.sum((y - A @ coef) ** 2))
        if cost < best[0]:
            best = (cost, np.array(sup), coef)
    return best


def test_top_s_matches_stable_sort():
    rng = np.random.Generator(np.random.PCG64(0))
    for trial in range(30):
        n = int(rng.integers(1, 200))
        s = int(rng.integers(1, n + 1))
        a = np.round(rng.standard_normal(n), 1)        # many ties
        sel, kth = oracle.top_s(a, s)
        order = np.lexsort((np.arange(n), -np.abs(a)))  # |a| descending, index ascending
        want = np.sort(order[:s])
        assert np.array_equal(sel, want)
        assert kth[0] == np.abs(a)[order[s - 1]]
        assert kth[1] == (np.abs(a)[order[s]] if s < n else 0.0)


def test_brute_force_noiseless_tiny():
    # NIHT is a local method: its recovery guarantee (Theorem 2) needs
    # gamma_2s <= 1/8, which tiny Gaussian matrices miss, so a few instances end
    # in a local minimum. Every output must still be stationary: the
    # least-squares solution on its own support.
    hits = 0
    trials = 40
    for seed in range(trials):
        p = synth.tiny(14, 16, 2, seed)
        phi = p.phi.astype(np.float64)
        y = phi @ p.x_true
        cost, sup, _ = _brute_force(phi, y, 2)
        assert cost < 1e-20 and np.array_equal(sup, p.support)
        res = oracle.niht(phi, phi, y, 2, 300)
        nz = np.flatnonzero(res.x)
        assert len(nz) <= 2
        ls, *_ = np.linalg.lstsq(phi[:, res.support], y, rcond=None)
        assert np.allclose(res.x[res.support], ls, rtol=1e-8, atol=1e-12)
        if np.linalg.norm(res.x - p.x_true) < 1e-8 * np.linalg.norm(p.x_true):
            hits += 1
    assert hits >= 0.9 * trials, hits


def test_brute_force_noisy_tiny_cost_bounds():
    # NIHT's cost is never below the global optimum, its output is the
    # least-squares fit on its own support, and on well-determined tiny
    # instances it usually is the global optimum
    equal = 0
    trials = 30
    for seed in range(trials):
        p = synth.tiny(16, 16, 2, 100 + seed, snr_db=20.0)
        phi = p.phi.astype(np.float64)
        y = p.y.astype(np.float64)
        cost, sup, _ = _brute_force(phi, y, 2)
        res = oracle.niht(phi, phi, y, 2, 400)
        c_niht = float(np.sum((y - phi @ res.x) ** 2))
        assert c_niht >= cost * (1 - 1e-9)
        ls, *_ = np.linalg.lstsq(phi[:, res.support], y, rcond=None)
        assert np.allclose(res.x[res.support], ls, rtol=1e-8, atol=1e-12)
        if c_niht <= cost * (1 + 1e-6):
            equal += 1
            assert np.array_equal(res.support, sup)
    assert equal >= 0.85 * trials, equal


def test_exact_recovery_gaussian():
    # noiseless s-sparse x from Gaussian Phi: the support is found and x is the
    # least-squares solution on it (y is stored in binary32, so "exact" means that)
    p = synth.gaussian(256, 1024, 16, seed=5, values="normal")
    phi = p.phi.astype(np.float64)
    y = p.y.astype(np.float64)
    res = oracle.niht(phi, phi, y, 16, 200)
    assert np.array_equal(res.support, p.support)
    ls, *_ = np.linalg.lstsq(phi[:, p.support], y, rcond=None)
    want = np.zeros(1024)
    want[p.support] = ls
    assert np.linalg.norm(res.x - want) <= 1e-10 * np.linalg.norm(want)
    assert np.linalg.norm(res.x - p.x_true) <= 1e-6 * np.linalg.norm(p.x_true)


def test_sparsity_and_step_size_bounds():
    p = synth.gaussian(64, 256, 8, seed=11, snr_db=20.0)
    phi = p.phi.astype(np.float64)
    y = p.y.astype(np.float64)
    res = oracle.niht(phi, phi, y, 8, 60, trace="x")
    tr = res.trace
    T = res.iters_run
    assert T > 5
    for t in range(1, T + 1):
        x = tr["x"][t]
        assert np.count_nonzero(x) <= 8
        assert set(np.flatnonzero(x)) <= set(tr["support"][t])
        # mu of iteration t was computed on the support of iteration t-1
        G = tr["support"][t - 1]
        sv = np.linalg.svd(phi[:, G], compute_uv=False)
        mu = tr["mu"][t]
        assert mu <= (1 / sv[-1] ** 2) * (1 + 1e-10)
        if tr["bt"][t] == 0:
            assert mu >= (1 / sv[0] ** 2) * (1 - 1e-10)


def _backtracking_instance():
    # a hard instance (many nonzeros, equal magnitudes) where shrinks occur
    for seed in range(40):
        p = synth.gaussian(48, 128, 12, seed=300 + seed, values="ones", snr_db=10.0)
        phi = p.phi.astype(np.float64)
        y = p.y.astype(np.float64)
        res = oracle.niht(phi, phi, y, 12, 80, trace="x")
        if res.backtracks > 0:
            return phi, y, res
    pytest.fail("no backtracking instance found")


def test_backtracking_condition_holds_on_support_change():
    phi, y, res = _backtracking_instance()
    tr = res.trace
    c = 0.01
    checked = 0
    for t in range(1, res.iters_run + 1):
        if np.array_equal(tr["support"][t], tr["support"][t - 1]):
            continue
        d = tr["x"][t] - tr["x"][t - 1]
        omega = np.dot(d, d) / np.dot(phi @ d, phi @ d)
        assert tr["mu"][t] <= (1 - c) * omega * (1 + 1e-10)
        checked += 1
    assert checked > 0


def test_cost_non_increasing_with_same_matrix():
    # Theorem 3 with Q1 = Q2: the majorisation argument gives monotone descent
    for seed in range(5):
        p = synth.gaussian(96, 384, 10, seed=50 + seed, snr_db=15.0)
        phi = p.phi.astype(np.float64)
        y = p.y.astype(np.float64)
        res = oracle.niht(phi, phi, y, 10, 100, trace=True)
        r2 = res.trace["resid2"][1:]
        assert np.all(np.diff(r2) <= 1e-10 * r2[:-1] + 1e-14), np.diff(r2).max()
        # and with a quantized matrix used for both products
        codes, c = oracle.quantize(p.phi, 4, seed=seed, stream=0)
        A = oracle.dequantize(codes, 4, c)
        res = oracle.niht(A, A, y, 10, 100, trace=True)
        r2 = res.trace["resid2"][1:]
        assert np.all(np.diff(r2) <= 1e-10 * r2[:-1] + 1e-14)


def test_double_sampling_gradient_is_unbiased():
    # E[Q1^T (Q(y) - Q2 x)] = Phi^T (y - Phi x) with independent Q1, Q2, Q(y) (Section III-A)
    p = synth.gaussian(32, 40, 4, seed=2, snr_db=20.0)
    phi = p.phi.astype(np.float64)
    y = p.y.astype(np.float64)
    x = p.x_true * 0.7
    exact = phi.T @ (y - phi @ x)
    bits = 2
    draws = []
    for seed in range(1500):
        c1, sphi = oracle.quantize(p.phi, bits, seed=seed, stream=0)
        c2, _ = oracle.quantize(p.phi, bits, seed=seed, stream=1, scale=sphi)
        cy, sy = oracle.quantize(p.y, bits, seed=seed, stream=2)
        A1 = oracle.dequantize(c1, bits, sphi)
        A2 = oracle.dequantize(c2, bits, sphi)
        yq = oracle.dequantize(cy, bits, sy)
        draws.append(oracle.gemv_t(A1, yq - A2 @ x))
    draws = np.array(draws)
    mean = draws.mean(axis=0)
    se = draws.std(axis=0, ddof=1) / np.sqrt(len(draws))
    z = np.abs(mean - exact) / se
    assert np.max(z) < 5.0, np.max(z)
    # the same matrix twice (no double sampling) is biased by the quantizer's variance
    biased = []
    for seed in range(1500):
        c1, sphi = oracle.quantize(p.phi, bits, seed=seed, stream=0)
        cy, sy = oracle.quantize(p.y, bits, seed=seed, stream=2)
        A1 = oracle.dequantize(c1, bits, sphi)
        yq = oracle.dequantize(cy, bits, sy)
        biased.append(oracle.gemv_t(A1, yq - A1 @ x))
    biased = np.array(biased)
    zb = np.abs(biased.mean(axis=0) - exact) / (biased.std(axis=0, ddof=1) / np.sqrt(len(biased)))
    assert np.max(zb) > 5.0


def test_qiht_approaches_niht_with_many_bits():
    p = synth.gaussian(128, 512, 8, seed=9, snr_db=30.0)
    ref = oracle.niht(p.phi, p.phi, p.y, 8, 150)
    errs = []
    for bits in (4, 8, 12, 16):
        res, _ = oracle.qiht(p.phi, p.y, 8, 150, bits_phi=bits, bits_y=bits, seed=1)
        errs.append(np.linalg.norm(res.x - ref.x) / np.linalg.norm(ref.x))
    assert errs[-1] < 1e-3
    assert errs[-1] < errs[0]
    assert errs[2] < errs[0]


def test_qiht_small_noiseless_recovers_support():
    p = synth.small_noiseless(0)
    res, q = oracle.qiht(p.phi, p.y, p.s, 200, bits_phi=8, bits_y=8, seed=0, trace=True)
    assert res.status == oracle.OK
    assert np.array_equal(res.support, p.support)
    rel = np.linalg.norm(res.x - p.x_true) / np.linalg.norm(p.x_true)
    assert rel < 0.05


def test_degenerate_zero_observation_stops():
    p = synth.gaussian(32, 64, 4, seed=1)
    res = oracle.niht(p.phi, p.phi, np.zeros(32), 4, 10)
    assert res.status == oracle.OK and res.iters_run == 0
    assert np.all(res.x == 0)


def test_argument_errors():
    A = np.zeros((4, 8))
    assert oracle.niht(A, A, np.zeros(4), 9, 3).status == oracle.ERR_ARG   # s > n
    assert oracle.niht(A, A, np.zeros(4), 5, 3).status == oracle.ERR_ARG   # s > m


def test_gradient_uses_first_matrix_and_step_uses_second():
    # Algorithm 2: g is formed with the first quantization and mu with the
    # second. With A1 = 2 A2, g doubles while mu (a ratio in A2 only) does not
    # change, so the first iterate H_s(0 + mu g) doubles exactly.
    p = synth.gaussian(40, 120, 5, seed=4, snr_db=20.0)
    A2 = p.phi.astype(np.float64)
    y = p.y.astype(np.float64)
    one = oracle.niht(A2, A2, y, 5, 1)
    two = oracle.niht(2.0 * A2, A2, y, 5, 1)
    assert np.array_equal(one.support, two.support)
    assert np.array_equal(2.0 * one.x, two.x)


# ---- fresh realizations per iteration (Algorithm 2 as written: 2n* matrices, n* observations) ----

def test_fresh_realizations_are_distinct_streams():
    T = 400
    phis = [oracle.phi_stream(k) for k in range(1, 2 * T + 1)]
    ys = [oracle.y_stream(t) for t in range(1, T + 1)]
    assert phis[:2] == [0, 1] and ys[0] == 2          # the first realizations are the fixed ones
    assert len(set(phis)) == len(phis) and len(set(ys)) == len(ys)
    assert not set(phis) & set(ys)


def test_fresh_gradient_is_unbiased_over_iterations():
    # one seed, the gradients Phi-hat_{2t-1}^T (y-hat_t - Phi-hat_{2t} x) of iterations t = 1..T at a
    # fixed x are independent draws whose mean is Phi^T (y - Phi x) (the double-sampling identity
    # stated before Algorithm 2)
    p = synth.gaussian(24, 32, 3, seed=5, snr_db=20.0)
    phi = p.phi.astype(np.float64)
    x = p.x_true * 0.6
    exact = phi.T @ (p.y.astype(np.float64) - phi @ x)
    bits, seed = 2, 77
    _, sphi = oracle.quantize(p.phi, bits, seed, 0)
    _, sy = oracle.quantize(p.y, bits, seed, 2)
    draws = []
    for t in range(1, 1201):
        c1, _ = oracle.quantize(p.phi, bits, seed, oracle.phi_stream(2 * t - 1), sphi)
        c2, _ = oracle.quantize(p.phi, bits, seed, oracle.phi_stream(2 * t), sphi)
        cy, _ = oracle.quantize(p.y, bits, seed, oracle.y_stream(t), sy)
        A1, A2 = oracle.dequantize(c1, bits, sphi), oracle.dequantize(c2, bits, sphi)
        draws.append(oracle.gemv_t(A1, oracle.dequantize(cy, bits, sy) - A2 @ x))
    draws = np.array(draws)
    z = np.abs(draws.mean(axis=0) - exact) / (draws.std(axis=0, ddof=1) / np.sqrt(len(draws)))
    assert np.max(z) < 5.0, np.max(z)


def test_fresh_first_iteration_is_the_fixed_one():
    # iteration 1 uses Phi-hat_1, Phi-hat_2 and y-hat_1 in both modes
    p = synth.gaussian(96, 384, 6, seed=12, snr_db=25.0)
    fx, _ = oracle.qiht(p.phi, p.y, p.s, 1, bits_phi=4, bits_y=4, seed=3, trace=True)
    fr, _ = oracle.qiht_fresh(p.phi, p.y, p.s, 1, bits_phi=4, bits_y=4, seed=3, trace=True)
    assert np.array_equal(fx.trace["support"], fr.trace["support"])
    assert np.array_equal(fx.x, fr.x) and fx.trace["mu"][1] == fr.trace["mu"][1]
    # and later iterations draw new realizations
    fx, _ = oracle.qiht(p.phi, p.y, p.s, 6, bits_phi=4, bits_y=4, seed=3, trace=True)
    fr, _ = oracle.qiht_fresh(p.phi, p.y, p.s, 6, bits_phi=4, bits_y=4, seed=3, trace=True)
    assert not np.array_equal(fx.trace["resid2"][2:], fr.trace["resid2"][2:])


def test_fresh_noiseless_recovers_and_approaches_niht_with_many_bits():
    p = synth.gaussian(128, 512, 8, seed=4)
    res, _ = oracle.qiht_fresh(p.phi, p.y, 8, 80, bits_phi=8, bits_y=8, seed=1)
    assert res.status == oracle.OK and np.array_equal(res.support, p.support)
    assert np.linalg.norm(res.x - p.x_true) / np.linalg.norm(p.x_true) < 0.05
    ref = oracle.niht(p.phi, p.phi, p.y, 8, 60)
    r16, _ = oracle.qiht_fresh(p.phi, p.y, 8, 60, bits_phi=16, bits_y=16, seed=2)
    assert np.linalg.norm(r16.x - ref.x) / np.linalg.norm(ref.x) < 1e-3
