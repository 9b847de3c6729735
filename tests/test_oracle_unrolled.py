"""Pins for the oracle of K unrolled QIHT iterations and their adjoint (oracle/unrolled.py).

The adjoint is checked against central finite differences of the forward map in FP64
(step 1e-6, directional derivatives along random directions and single coordinates), at
the problem size m = 64, n = 256, with the support masks of every step unchanged at both
perturbed points (the map is differentiable there). A planted mistake in the adjoint (a
dropped term of the step size's derivative) fails the same check."""
import numpy as np
import pytest

import oracle
from oracle import unrolled
import synth


def _problem(seed=0, m=64, n=256, s=8, bits=4):
    rng = np.random.Generator(np.random.PCG64(seed))
    phi = (rng.standard_normal((m, n)) / np.sqrt(m)).astype(np.float32)
    x = np.zeros(n)
    sup = rng.choice(n, s, replace=False)
    x[sup] = rng.standard_normal(s)
    mag = rng.uniform(0.9, 1.1, m)
    ph = rng.uniform(-0.1, 0.1, m)
    a, b = mag * np.cos(ph), mag * np.sin(ph)
    clean = unrolled.stacked(phi.astype(np.float64), a, b) @ x
    y = clean + np.sqrt(clean @ clean / (2 * m * 1e3)) * rng.standard_normal(2 * m)
    c1, sc = oracle.quantize(phi, bits, seed, 0)
    c2, _ = oracle.quantize(phi, bits, seed, 1, sc)
    P1, P2 = oracle.dequantize(c1, bits, sc), oracle.dequantize(c2, bits, sc)
    return P1, P2, y, a, b, x, s


def _masks(steps):
    return [tuple(st.Gn) for st in steps] + [tuple(steps[0].G)]


def _fd_check(P1, P2, y, a, b, x, s, K, which, direction, eps=1e-6, bwd=unrolled.backward):
    L0, gy, ga, gb, _, steps = unrolled.loss_and_grads(P1, P2, y, a, b, s, K, x)
    if bwd is not unrolled.backward:
        xK, st2 = unrolled.forward(P1, P2, y, a, b, s, K)
        gy, ga, gb = bwd(P1, P2, a, b, st2, 2.0 * (xK - x))
    args = {"y": y, "a": a, "b": b}
    grads = {"y": gy, "a": ga, "b": gb}
    plus, minus = dict(args), dict(args)
    plus[which] = args[which] + eps * direction
    minus[which] = args[which] - eps * direction
    Lp, *_, sp = unrolled.loss_and_grads(P1, P2, plus["y"], plus["a"], plus["b"], s, K, x)
    Lm, *_, sm = unrolled.loss_and_grads(P1, P2, minus["y"], minus["a"], minus["b"], s, K, x)
    assert _masks(sp) == _masks(steps) == _masks(sm), "a support changed under the perturbation"
    fd = (Lp - Lm) / (2 * eps)
    an = float(grads[which] @ direction)
    return fd, an


@pytest.mark.parametrize("which", ["y", "a", "b"])
@pytest.mark.parametrize("K", [1, 3, 8])
def test_adjoint_matches_central_differences(which, K):
    P1, P2, y, a, b, x, s = _problem(seed=K)
    rng = np.random.Generator(np.random.PCG64(100 + K))
    size = y.size if which == "y" else a.size
    for _ in range(3):
        d = rng.standard_normal(size)
        fd, an = _fd_check(P1, P2, y, a, b, x, s, K, which, d)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (which, K, fd, an)


def test_adjoint_single_coordinates():
    P1, P2, y, a, b, x, s = _problem(seed=7)
    for which, idx in (("y", [0, 5, 70, 127]), ("a", [1, 33, 63]), ("b", [0, 40])):
        size = y.size if which == "y" else a.size
        for i in idx:
            e = np.zeros(size)
            e[i] = 1.0
            fd, an = _fd_check(P1, P2, y, a, b, x, s, 5, which, e)
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (which, i, fd, an)


def test_forward_is_the_iteration_of_algorithm_2_without_backtracking():
    # with gains (1, 0) and one quantized matrix twice, one unrolled step equals the first
    # iteration of the oracle's Algorithm 2 whenever that iteration did not backtrack
    P1, P2, y, a, b, x, s = _problem(seed=3)
    m = P1.shape[0]
    ones, zeros = np.ones(m), np.zeros(m)
    yt = y[:m]
    xK, steps = unrolled.forward(P1, P2, np.concatenate([yt, np.zeros(m)]), ones, zeros, s, 1)
    ref = oracle.niht(P1, P2, yt, s, 1, trace=True)
    assert ref.trace["bt"][1] == 0
    assert np.array_equal(np.sort(np.flatnonzero(xK)), np.sort(ref.support))
    assert np.allclose(xK, ref.x, rtol=1e-12, atol=1e-14)


def test_stacked_is_the_complex_gain():
    # [diag(a); diag(b)] Phi x is the real and imaginary part of g * (Phi x), g = a + i b
    rng = np.random.Generator(np.random.PCG64(11))
    m, n = 9, 7
    phi = rng.standard_normal((m, n))
    a, b, x = rng.standard_normal(m), rng.standard_normal(m), rng.standard_normal(n)
    z = (a + 1j * b) * (phi @ x)
    assert np.allclose(unrolled.stacked(phi, a, b) @ x, np.concatenate([z.real, z.imag]), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("seed,bits", [(4, 4), (7, 4), (5, 8), (9, 2)])
def test_forward_with_gains_is_algorithm_2_on_the_stacked_system(seed, bits):
    # with the gains of the workload and the two different quantizations, one unrolled step
    # equals the first iteration of the oracle's Algorithm 2 (C) on A_i = [diag(a); diag(b)] Q_i
    # when that iteration did not backtrack (later iterations of these instances do, which the
    # unrolled map leaves out)
    P1, P2, y, a, b, x, s = _problem(seed=seed, bits=bits)
    A1, A2 = unrolled.stacked(P1, a, b), unrolled.stacked(P2, a, b)
    ref = oracle.niht(A1, A2, y, s, 1, trace=True)
    assert ref.trace["bt"][1] == 0
    xK, steps = unrolled.forward(P1, P2, y, a, b, s, 1)
    assert np.array_equal(np.flatnonzero(xK), np.sort(ref.support))
    assert np.allclose(xK, ref.x, rtol=1e-12, atol=1e-14)
    assert abs(steps[0].mu - ref.trace["mu"][1]) <= 1e-12 * steps[0].mu


def test_dropped_term_is_caught():
    # a planted mistake: the step size treated as a constant (its derivative dropped)
    def bad_backward(Phi1, Phi2, a, b, steps, xbar):
        fixed = [unrolled.Step(**{**st.__dict__, "D": 0.0}) for st in steps]
        return unrolled.backward(Phi1, Phi2, a, b, fixed, xbar)
    P1, P2, y, a, b, x, s = _problem(seed=2)
    d = np.random.Generator(np.random.PCG64(5)).standard_normal(y.size)
    fd, an = _fd_check(P1, P2, y, a, b, x, s, 4, "y", d, bwd=bad_backward)
    assert abs(fd - an) > 1e-4 * max(1.0, abs(fd))
