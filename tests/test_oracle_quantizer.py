"""Pins for the oracle's stochastic quantizer Q(v, b) (Section III-A) and its
scale c_v = max |v| (Appendix, quantization-error lemma).

Each check is fixed by the paper's definition or by mathematics, not by the
oracle itself: codes on the 2^b grid, deterministic results where the value is
a grid point, unbiasedness E[Q(v)] = v, the rounding-up probability, the error
bound of the quantization lemma, and independence of the random numbers from
the storage layout. The odd grid of 2^(b-1) + 1 levels (the Appendix's remark on
fixed-point hardware) is pinned by its level set, its exact zero, the ternary
case b = 2 worked by hand, and the lemma's bound, which that grid's spacing gives.
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


@pytest.mark.parametrize("odd", [False, True])
@pytest.mark.parametrize("bits", [2, 4, 8])
def test_unbiased(bits, odd):
    # E[Q(v)] = v (Section III-A): mean over many independent draws within 5 sigma
    v = synth.random_floats(48, seed=20 + bits)
    v[0] = np.abs(v).max() * 1.5          # fixes the scale
    reps = 4000
    mat = np.repeat(v[:, None], reps, axis=1)
    codes, c = oracle.quantize(mat, bits, seed=123, stream=0, odd=odd)
    deq = oracle.dequantize(codes, bits, c, odd=odd)
    mean = deq.mean(axis=1)
    lm1 = 2 ** (bits - 1) if odd else 2**bits - 1
    spacing = 2.0 * c / lm1
    t = (v.astype(np.float64) / c + 1) * lm1 / 2
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


# ---- the odd grid of the Appendix's remark: 2^(b-1) + 1 levels, spacing 1/2^(b-2) ----

@pytest.mark.parametrize("bits", [2, 4, 8])
def test_odd_grid_codes_on_grid(bits):
    nlev = 2 ** (bits - 1) + 1
    assert oracle.levels(bits, odd=True) == nlev and oracle.levels(bits) == 2**bits
    v = synth.random_floats((37, 53), seed=40 + bits)
    v[0, 0] = np.abs(v).max()
    v[0, 1] = -v[0, 0]
    codes, c = oracle.quantize(v, bits, seed=6, stream=1, odd=True)
    assert codes.max() <= nlev - 1 and codes.min() >= 0
    deq = oracle.dequantize(codes, bits, c, odd=True)
    # levels -1, -1 + 1/2^(b-2), ..., 1 (times c), written from the remark's spacing
    grid = c * (-1.0 + np.arange(nlev) / 2.0 ** (bits - 2))
    assert grid[-1] == c
    assert np.all(np.isin(np.round(deq, 12), np.round(grid, 12)))
    # each value goes to one of the two grid points around it
    assert np.all(np.abs(deq - v) <= c / 2.0 ** (bits - 2) * (1 + 1e-6))
    # +-c go to the end levels
    assert codes[0, 0] == nlev - 1 and codes[0, 1] == 0


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_odd_grid_has_an_exact_zero(bits):
    # 0 is a level of the odd grid: zero inputs quantize to it for every random number,
    # whereas the 2^b grid (an even number of levels) has no zero level
    v = np.zeros(4000, dtype=np.float32)
    v[0] = np.float32(2.5)                     # sets c
    codes, c = oracle.quantize(v, bits, seed=11, stream=0, odd=True)
    assert np.all(codes[1:] == 2 ** (bits - 2))
    assert np.all(oracle.dequantize(codes[1:], bits, c, odd=True) == 0.0)
    codes_e, _ = oracle.quantize(v, bits, seed=11, stream=0)
    deq_e = oracle.dequantize(codes_e[1:], bits, c)
    assert np.all(deq_e != 0.0) and abs(deq_e.mean()) < 0.1 * c


def test_odd_grid_two_bits_is_ternary():
    # b = 2: levels {-c, 0, c}. v = c/4 lies between 0 and c with f = 1/4 exactly, so its
    # code is 1 + (u < 1/4) for the element's own uniform u (the generator is pinned
    # separately against Philox4x32-10)
    n = 3000
    v = np.full(n, 0.25, dtype=np.float32)
    v[0] = np.float32(1.0)
    seed, stream = 21, 2
    codes, c = oracle.quantize(v, 2, seed=seed, stream=stream, odd=True)
    assert c == 1.0 and codes[0] == 2
    u = np.array([oracle.uniform(seed, stream, e) for e in range(n)])
    assert np.array_equal(codes[1:], 1 + (u[1:] < 0.25))
    assert np.array_equal(np.unique(oracle.dequantize(codes, 2, c, odd=True)), [0.0, 1.0])


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_odd_grid_error_bound_of_quantization_lemma(bits):
    # The lemma's bound E||Q(v, b) - v||_2 <= c_v sqrt(M) / 2^(b-1) comes from the odd grid's
    # spacing 1/2^(b-2): half a spacing squared, summed over M entries. It holds here, and the
    # per-draw error stays below the worst case sqrt(M) * spacing / 2.
    M = 512
    v = synth.random_floats(M, seed=60 + bits)
    c = float(np.abs(v).max())
    errs = []
    for seed in range(60):
        codes, _ = oracle.quantize(v, bits, seed=seed, stream=2, odd=True)
        errs.append(np.linalg.norm(oracle.dequantize(codes, bits, c, odd=True) - v))
    assert max(errs) <= c * np.sqrt(M) / 2 ** (bits - 1) * (1 + 1e-9)
    e = np.mean(errs)
    assert e <= c * np.sqrt(M) / 2 ** (bits - 1)
    assert e > 0.1 * c * np.sqrt(M) / 2 ** (bits - 1)
