"""Pins for the oracle's stochastic quantizer Q(v, b) (Section III-A) and its
scale c_v = max |v| (Appendix, quantization-error lemma).

Each check is fixed by the paper's definition or by mathematics, not by the
oracle itself: codes on the 2^b grid, deterministic results where the value is
a grid point, unbiasedness E[Q(v)] = v, the rounding-up probability, the error
bound of the quantization lemma, and independence of the random numbers from
the storage layout.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_codes_on_grid_and_scale(bits):
    v = synth.random_floats((37, 53), seed=bits)
    codes, c = oracle.quantize(v, bits, seed=5, stream=0)
    assert c == float(np.abs(v).max())
    assert codes.min() >= 0 and codes.max() <= 2**bits - 1
    deq = oracle.dequantize(codes, bits, c)
    levels = c * (-1.0 + 2.0 * np.arange(2**bits) / (2**bits - 1))
    assert np.all(np.isin(np.round(deq, 12), np.round(levels, 12)))
    # every value is rounded to one of the two grid points around it
    t = (v.astype(np.float64) / c + 1.0) * (2**bits - 1) / 2
    assert np.all(np.abs(codes - t) < 1.0 + 1e-5)


def test_absmax_and_nonfinite():
    v = synth.random_floats(1000, seed=1)
    c, bad = oracle.absmax(v)
    assert c == float(np.max(np.abs(v))) and bad == 0
    v[17] = np.nan
    v[99] = np.inf
    _, bad = oracle.absmax(v)
    assert bad == 2


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_endpoints_and_exact_grid_points_are_deterministic(bits):
    L = 2**bits
    # +-c quantize to the end codes for every random number
    v = np.array([1.0, -1.0] * 500, dtype=np.float32) * np.float32(3.5)
    codes, _ = oracle.quantize(v, bits, seed=9, stream=0)
    assert np.all(codes[0::2] == L - 1) and np.all(codes[1::2] == 0)
    # values whose grid position t is an exact integer in binary32 arithmetic
    half = np.float32((L - 1) / 2)
    cands = []
    for k in range(L):
        vt = np.float32(np.float32(2 * k) / np.float32(L - 1)) - np.float32(1)
        t = (vt + np.float32(1)) * half
        if t == np.float32(k):
            cands.append((k, vt))
    assert cands, "no exact grid points found"
    vals = np.array([vt for _, vt in cands] + [np.float32(1.0)], dtype=np.float32)
    reps = np.tile(vals, 300)
    codes, c = oracle.quantize(reps, bits, seed=4, stream=1)
    assert c == 1.0
    want = np.tile(np.array([k for k, _ in cands] + [L - 1]), 300)
    assert np.array_equal(codes, want)


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_unbiased(bits):
    # E[Q(v)] = v (Section III-A): mean over many independent draws within 5 sigma
    v = synth.random_floats(48, seed=20 + bits)
    v[0] = np.abs(v).max() * 1.5          # fixes the scale
    reps = 4000
    mat = np.repeat(v[:, None], reps, axis=1)
    codes, c = oracle.quantize(mat, bits, seed=123, stream=0)
    deq = oracle.dequantize(codes, bits, c)
    mean = deq.mean(axis=1)
    spacing = 2.0 * c / (2**bits - 1)
    t = (v.astype(np.float64) / c + 1) * (2**bits - 1) / 2
    f = t - np.floor(t)
    sd = spacing * np.sqrt(f * (1 - f) / reps) + 1e-12
    z = np.abs(mean - v) / sd
    assert np.all((z < 5.0) | (np.abs(mean - v) < 1e-6 * c)), z.max()


def test_round_up_probability_equals_fraction():
    # P(code = i + 1) = f = t - i; a reversed comparison would give 1 - f
    bits = 4
    L = 2**bits
    c = np.float32(1.0)
    for target_f in (0.1, 0.3, 0.75):
        t = np.float32(5 + target_f)
        vt = np.float32(t / np.float32((L - 1) / 2) - np.float32(1))
        t_eff = float((vt + np.float32(1)) * np.float32((L - 1) / 2))
        f = t_eff - 5
        reps = 20000
        v = np.full(reps, vt, dtype=np.float32)
        v[0] = c
        codes, _ = oracle.quantize(v, bits, seed=77, stream=0)
        frac = np.mean(codes[1:] == 6)
        assert np.all(np.isin(codes[1:], [5, 6]))
        assert abs(frac - f) < 5 * np.sqrt(f * (1 - f) / reps)


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_error_bound_of_quantization_lemma(bits):
    # E||Q(v, b) - v||_2 <= c_v sqrt(M) / 2^(b-1) (Appendix, quantization lemma);
    # with the 2^b-level grid the tighter bound c_v sqrt(M) / (2^b - 1) also holds.
    M = 512
    v = synth.random_floats(M, seed=bits)
    c = float(np.abs(v).max())
    errs = []
    for seed in range(60):
        codes, _ = oracle.quantize(v, bits, seed=seed, stream=2)
        errs.append(np.linalg.norm(oracle.dequantize(codes, bits, c) - v))
    e = np.mean(errs)
    assert e <= c * np.sqrt(M) / 2 ** (bits - 1)
    assert e <= c * np.sqrt(M) / (2**bits - 1)
    # and not trivially small: the rounding really is stochastic
    assert e > 0.1 * c * np.sqrt(M) / (2**bits - 1)


def test_codes_depend_only_on_position():
    # a block quantized at its position equals the same block of the whole matrix
    v = synth.random_floats((40, 30), seed=8)
    full, c = oracle.quantize(v, 8, seed=3, stream=1)
    blk, _ = oracle.quantize(v[7:19, 11:29], 8, seed=3, stream=1, scale=c, row0=7, col0=11, rows_total=40)
    assert np.array_equal(blk, full[7:19, 11:29])
    # a column quantized as a vector uses the same numbering
    col, _ = oracle.quantize(v[:, 5], 8, seed=3, stream=1, scale=c, col0=5, rows_total=40)
    assert np.array_equal(col, full[:, 5])


def test_double_sampling_streams_are_independent():
    v = synth.random_floats((64, 64), seed=2)
    c1, c = oracle.quantize(v, 2, seed=1, stream=0)
    c2, _ = oracle.quantize(v, 2, seed=1, stream=1)
    d1 = oracle.dequantize(c1, 2, c) - v
    d2 = oracle.dequantize(c2, 2, c) - v
    rho = np.corrcoef(d1.ravel(), d2.ravel())[0, 1]
    assert abs(rho) < 5 / np.sqrt(v.size)
    assert not np.array_equal(c1, c2)


def test_zero_scale_gives_zero_values():
    v = np.zeros(100, dtype=np.float32)
    codes, c = oracle.quantize(v, 4, seed=0, stream=0)
    assert c == 0.0
    assert np.all(oracle.dequantize(codes, 4, c) == 0.0)
