"""The quantizer's division v / c by the scale c (one divisor for a whole quantization), checked on
the CPU in exact rational arithmetic.

The kernels compute the binary32 decision t = (v / c + 1) (L - 1) / 2 with each operation
correctly rounded. For v / c they use Markstein's FMA division: y = RN(1/c) once, then
q = RN(v y), r = RN(v - c q) (one FMA) and RN(q + r y) (another). This test replays those steps
with exact fractions rounded once each to binary32, as the FMA does, on random and edge-case
pairs with |v| <= c, and checks:
- that the result equals RN(v / c) wherever |v / c| >= 2^-25;
- that below that, where 1 + v/c rounds to 1, the decision t is the same either way.
"""
from fractions import Fraction

import numpy as np

_MIN_NORMAL_EXP = -126


def rn32(x: Fraction) -> Fraction:
    """x rounded to the nearest binary32 (ties to even), subnormals included, as a Fraction."""
    if x == 0:
        return Fraction(0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, _MIN_NORMAL_EXP)                 # below 2^-126 the spacing stays 2^-149
    ulp = Fraction(2) ** (e - 23)
    m = a / ulp
    lo = m.numerator // m.denominator
    rem = m - lo
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and lo % 2 == 1):
        lo += 1
    return sign * lo * ulp


def f32(x) -> Fraction:
    return Fraction(float(np.float32(x)))


def is_f32(x: Fraction) -> bool:
    return rn32(x) == x


def decision(q: Fraction, half: Fraction) -> Fraction:
    return rn32(rn32(q + 1) * half)


def _pairs(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    cs = np.concatenate([rng.uniform(1e-3, 1e3, n // 2), 10.0 ** rng.uniform(-30, 30, n // 2)]).astype(np.float32)
    cs = np.concatenate([cs, np.float32([1.0, 0.1, 3.0, 0.99999994, 1.0000001, 2.0**-100, 2.0**100])])
    out = []
    for c in cs:
        c = np.float32(c)
        for frac in (rng.uniform(-1, 1), rng.uniform(-1e-6, 1e-6), 1.0, -1.0, rng.uniform(-1e-30, 1e-30)):
            v = np.float32(np.clip(np.float32(frac) * c, -c, c))
            out.append((v, c))
        # a subnormal v
        out.append((np.float32(1e-45), c))
    return out


def test_markstein_division_matches_correct_rounding():
    half = Fraction(255, 2)                     # 8 bits: (L - 1) / 2
    small = 0
    for v32, c32 in _pairs(1500, 7):
        v, c = f32(v32), f32(c32)
        y = rn32(1 / c)
        q = rn32(v * y)
        r = rn32(v - c * q)                     # the FMA: exact product and sum, one rounding
        q2 = rn32(q + r * y)
        ref = rn32(v / c)
        if abs(v / c) >= Fraction(2) ** -25:
            assert q2 == ref, (v32, c32, float(q2), float(ref))
        else:
            small += 1
            assert abs(q2) < Fraction(2) ** -25
            assert decision(q2, half) == decision(ref, half)
    assert small > 0                            # tiny and subnormal quotients were covered


def test_rn32_agrees_with_numpy():
    rng = np.random.Generator(np.random.PCG64(3))
    for x in np.concatenate([rng.standard_normal(200) * 10.0 ** rng.uniform(-44, 37, 200), [1e-45, 3e-39, 1.5]]):
        assert rn32(Fraction(float(x))) == Fraction(float(np.float32(x))), x
