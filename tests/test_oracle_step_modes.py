"""Pins of the oracle's two step-size denominators and of its residual tolerance.

Algorithm 2 prints the step size mu = ||g_G||^2 / ((Phi_{2n-1})_G g_G)^T ((Phi_{2n})_G g_G):
the product of the images of g_G under two independent realizations of Q(Phi). The
oracle's default reading uses the forward square ||Q2_G g_G||^2 instead (positive by
construction); mu_mode "cross" computes the printed product and falls back to the forward
square when the product is not positive.

Pinned here against facts that do not come from the oracle itself:
  - with one realization used twice the two denominators are the same number, so the
    whole trajectory is bitwise the forward-square one;
  - with A1 = -A2 the product is -||A2_G g_G||^2 < 0: the fallback must engage;
  - the quantizer is unbiased and the two realizations are independent, so the product
    is an unbiased estimate of ||Phi_G g_G||^2, while the forward square is biased
    upwards by exactly sum_i sum_j g_j^2 Var(Q(Phi)_ij), Var = D^2 f (1 - f) for a
    value at fraction f of a grid step D (Section III-A, the quantizer's definition);
  - tol: on a noiseless instance with exact recovery the residual goes to zero, so a
    tiny tol stops the run early with x equal to the true signal; tol = 0 changes
    nothing; a tol between two residuals of the trace stops at the first iteration
    below it, with that iteration's iterate.
"""
import numpy as np

import oracle
import synth


def _instance(m=48, n=96, s=6, seed=3):
    p = synth.gaussian(m, n, s, seed=seed, snr_db=30.0)
    return p


def test_cross_equals_forward_with_one_realization():
    p = _instance()
    A = oracle.dequantize(*oracle.quantize(p.phi, 8, 5, 0)[:1], 8, oracle.quantize(p.phi, 8, 5, 0)[1])
    yq = p.y.astype(np.float64)
    a = oracle.niht(A, A, yq, p.s, 40, trace="x")
    b = oracle.niht(A, A, yq, p.s, 40, mu_mode="cross", trace="x")
    assert a.iters_run == b.iters_run == 40
    for k in ("support", "mu", "resid2", "x", "bt"):
        assert np.array_equal(a.trace[k], b.trace[k]), k
    assert not b.trace["mu_fallback"].any()


def test_cross_falls_back_when_not_positive():
    p = _instance(seed=4)
    A2 = p.phi.astype(np.float64)
    A1 = -A2
    rng = np.random.Generator(np.random.PCG64(1))
    sup = np.sort(rng.choice(p.n, p.s, replace=False)).astype(np.int32)
    g = rng.standard_normal(p.n)
    fwd = oracle.step_size(A1, A2, sup, g, "forward")
    cr = oracle.step_size(A1, A2, sup, g, "cross")
    assert cr["cross"] < 0 and cr["fallback"]
    assert cr["den"] == fwd["den"] and cr["num"] == fwd["num"]
    # inside the solve: the first iteration's step falls back, so its mu is the forward one
    r1 = oracle.niht(A1, A2, p.y, p.s, 1, mu_mode="cross", trace=True)
    r0 = oracle.niht(A1, A2, p.y, p.s, 1, trace=True)
    assert r1.trace["mu_fallback"][1] == 1
    assert r1.trace["mu"][1] == r0.trace["mu"][1]


def test_cross_is_unbiased_and_forward_square_carries_the_variance():
    # fixed Phi, support and g; many independent pairs (Q1, Q2) of 4-bit quantizations
    m, n, s, bits = 24, 40, 5, 4
    rng = np.random.Generator(np.random.PCG64(7))
    phi = (rng.standard_normal((m, n)) / np.sqrt(m)).astype(np.float32)
    sup = np.sort(rng.choice(n, s, replace=False)).astype(np.int32)
    g = np.zeros(n)
    g[sup] = rng.standard_normal(s)
    exact = float(np.sum((phi.astype(np.float64)[:, sup] @ g[sup]) ** 2))
    # variance of each quantized entry from the quantizer's definition (2^b levels on [-1, 1]
    # scaled by c = max |Phi|): a value at fraction f of a step D rounds up with probability f
    c = float(np.max(np.abs(phi)))
    L = 2**bits
    D = 2.0 * c / (L - 1)
    t = (phi.astype(np.float64) / c + 1.0) * (L - 1) / 2.0
    f = t - np.floor(t)
    var = D * D * f * (1.0 - f)
    bias = float(np.sum(var[:, sup] @ (g[sup] ** 2)))
    K = 3000
    cross, fwd = np.empty(K), np.empty(K)
    for k in range(K):
        c1, sc = oracle.quantize(phi, bits, 1000 + k, 0)
        c2, _ = oracle.quantize(phi, bits, 1000 + k, 1, sc)
        A1 = oracle.dequantize(c1, bits, sc)
        A2 = oracle.dequantize(c2, bits, sc)
        st = oracle.step_size(A1, A2, sup, g, "cross")
        cross[k] = st["cross"]
        fwd[k] = oracle.step_size(A1, A2, sup, g, "forward")["den"]
    se_c = cross.std(ddof=1) / np.sqrt(K)
    se_f = fwd.std(ddof=1) / np.sqrt(K)
    assert abs(cross.mean() - exact) <= 5 * se_c, (cross.mean(), exact, se_c)
    assert abs(fwd.mean() - (exact + bias)) <= 5 * se_f, (fwd.mean(), exact + bias, se_f)
    assert bias > 10 * se_f            # the forward square's bias is resolved by the sample


def test_tol_stops_exact_recovery_early():
    # noiseless Gaussian instance, unquantized (Algorithm 1): NIHT recovers x exactly, so the
    # residual falls to rounding level and a tiny tol ends the run before the iteration cap
    p = synth.small_noiseless(0)
    A = p.phi.astype(np.float64)
    y = A @ p.x_true
    full = oracle.niht(A, A, y, p.s, 200, trace=True)
    res = oracle.niht(A, A, y, p.s, 200, tol=1e-20, trace=True)
    assert res.iters_run < 200
    assert res.resid_norm2 <= 1e-20
    assert res.trace["resid2"][res.iters_run] <= 1e-20
    assert np.all(res.trace["resid2"][1:res.iters_run] > 1e-20)
    assert np.linalg.norm(res.x - p.x_true) <= 1e-8 * np.linalg.norm(p.x_true)
    assert full.iters_run == 200


def test_tol_zero_changes_nothing_and_between_residuals_stops_there():
    p = synth.gaussian(64, 200, 6, seed=9, snr_db=20.0)
    res0, _ = oracle.qiht(p.phi, p.y, p.s, 30, bits_phi=8, bits_y=8, seed=2, trace="x")
    resz, _ = oracle.qiht(p.phi, p.y, p.s, 30, bits_phi=8, bits_y=8, seed=2, trace="x", tol=0.0)
    assert np.array_equal(res0.x, resz.x) and res0.iters_run == resz.iters_run == 30
    r2 = res0.trace["resid2"]
    t0 = 4
    tol = 0.5 * (r2[t0] + min(r2[1:t0]))      # below every residual before t0, above r2[t0]
    assert r2[t0] < tol < min(r2[1:t0])
    rt, _ = oracle.qiht(p.phi, p.y, p.s, 30, bits_phi=8, bits_y=8, seed=2, trace="x", tol=tol)
    assert rt.iters_run == t0
    assert np.array_equal(rt.x, res0.trace["x"][t0])
    big, _ = oracle.qiht(p.phi, p.y, p.s, 30, bits_phi=8, bits_y=8, seed=2, tol=1e30)
    assert big.iters_run == 1
