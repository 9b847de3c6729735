"""Pins of the oracle's E4M3 rounding and of the three-term residual (the FP8 gradient).

E4M3 is the OCP 8-bit floating-point format with 4 exponent bits (bias 7), 3 fraction bits
and subnormals, whose largest finite value is 448; codes of at most 4 bits are exact in it
(Section III-A's b-bit levels are integers of at most 4 significant bits after centring).
The oracle rounds to it from the format's definition; these tests hold that rounding against
PyTorch's own float8_e4m3fn conversion and against facts of the format, and the three-term
representation against the error bound that the format's precision gives."""
import numpy as np
import pytest
import torch

import oracle


def _torch_e4m3(v):
    return torch.from_numpy(np.asarray(v, dtype=np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()


def _finite_values():
    """All non-negative finite E4M3 values from their bit fields (exponent, fraction)."""
    vals = [f / 8 * 2.0**-6 for f in range(8)]                          # zero and subnormals
    for E in range(1, 16):
        for f in range(8):
            if E == 15 and f == 7:
                continue                                                 # the NaN encoding
            vals.append((1 + f / 8) * 2.0 ** (E - 7))
    return np.array(vals)


def test_e4m3_matches_torch_cast():
    pos = _finite_values()
    mids = (pos[1:] + pos[:-1]) / 2                                      # exact ties
    rng = np.random.Generator(np.random.PCG64(3))
    rand = np.exp2(rng.uniform(-12.0, np.log2(440.0), 20000)).astype(np.float32).astype(np.float64)
    v = np.concatenate([pos, mids, rand, pos * 1.0000001, pos * 0.9999999])
    v = v[v <= 448.0]
    v = np.concatenate([v, -v])
    got = oracle.e4m3(v)
    ref = _torch_e4m3(v)
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, [(v[i], got[i], ref[i]) for i in bad[:5]]


def test_e4m3_format_facts():
    e = oracle.e4m3
    assert e(448.0) == 448.0 and e(460.0) == 448.0 and e(1e6) == 448.0 and e(-1e6) == -448.0   # saturation
    assert e(2.0**-9) == 2.0**-9                                         # smallest subnormal
    assert e(2.0**-10) == 0.0                                            # tie with zero: even
    assert e(3 * 2.0**-10) == 2.0**-8                                    # tie 1/8 and 2/8 of 2^-6: even
    assert e(1.0625) == 1.0 and e(1.1875) == 1.25                        # ties to the even fraction
    assert e(17.0) == 16.0 and e(19.0) == 20.0
    assert e(0.0) == 0.0
    # every odd integer up to 15 (the centred 4-bit codes) and every integer up to 16 is exact
    ints = np.arange(-16, 17, dtype=np.float64)
    assert np.array_equal(e(ints), ints)
    # 127 distinct non-negative finite values over a fine sweep
    sweep = np.exp2(np.linspace(-11.0, np.log2(448.0), 200001))
    assert np.unique(e(np.concatenate([[0.0], sweep]))).size == 127


def _wide(rng, m, scale_pow):
    mag = np.exp2(rng.uniform(-22.0, 0.0, m))
    r = rng.choice([-1.0, 1.0], m) * mag * 2.0**scale_pow
    r[rng.integers(m)] = 0.97 * 2.0**scale_pow                          # max near the top of its binade
    r[rng.integers(m)] = 0.0
    return r


@pytest.mark.parametrize("scale_pow", [-30, -3, 0, 5, 40])
def test_e4m3_terms_error_bound(scale_pow):
    # r' = r 2^-e with max |r'| in [2^7, 2^8): three terms carry r' to within
    # 2^-12 |r'| (each term keeps 4 significant bits of what is left) + 2^-10 (half the
    # smallest subnormal), and no term saturates
    rng = np.random.Generator(np.random.PCG64(scale_pow + 100))
    for _ in range(4):
        r = _wide(rng, 4096, scale_pow)
        out = oracle.e4m3_terms(r)
        e = np.frexp(np.abs(r).max())[1] - 8
        err = np.abs(ldexp(r - out, -e))
        assert np.all(err <= 2.0**-12 * np.abs(ldexp(r, -e)) + 2.0**-10), err.max()
        assert np.abs(ldexp(out, -e)).max() < 2.0**8
        # one term alone is coarse: the representation uses all three
        one = oracle.e4m3_terms(r, terms=1)
        assert np.abs(one - r).max() > np.abs(out - r).max()


def ldexp(a, e):
    return np.ldexp(a, e)


def test_e4m3_terms_exact_for_representable():
    # vectors whose scaled entries are E4M3 values come back unchanged, at any power-of-two scale
    rng = np.random.Generator(np.random.PCG64(9))
    pos = _finite_values()
    for k in (-40, -7, 0, 12):
        t = rng.choice(pos[pos < 256.0], 777) * rng.choice([-1.0, 1.0], 777)
        t[5] = 240.0                                                     # max in [2^7, 2^8)
        r = np.ldexp(t, k)
        assert np.array_equal(oracle.e4m3_terms(r), r)
    z = np.zeros(50)
    assert np.array_equal(oracle.e4m3_terms(z), z)


def test_grad_e4m3_solve_recovers_noiseless():
    # with Phi itself (no quantization) and no noise, the gradient's relative error shrinks with
    # the residual: the e4m3 mode still recovers x exactly (to rounding)
    rng = np.random.Generator(np.random.PCG64(4))
    m, n, s = 128, 256, 6
    phi = rng.standard_normal((m, n)) / np.sqrt(m)
    x = np.zeros(n)
    sup = np.sort(rng.choice(n, s, replace=False))
    x[sup] = rng.choice([-1.0, 1.0], s) * rng.uniform(0.5, 1.5, s)
    y = phi @ x
    res = oracle.niht(phi, phi, y, s, 200, grad_e4m3=True)
    assert np.array_equal(res.support, sup)
    assert np.linalg.norm(res.x - x) <= 1e-9 * np.linalg.norm(x)
    # and its path differs from the exact gradient's (the mode is in effect)
    ex = oracle.niht(phi, phi, y, s, 3, trace=True)
    e8 = oracle.niht(phi, phi, y, s, 3, grad_e4m3=True, trace=True)
    assert not np.array_equal(ex.trace["mu"], e8.trace["mu"])
