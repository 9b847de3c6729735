"""Kernel-level parity through the C ABI: qiht_gemv_t (Q^T r), qiht_gemv_cols
(Q[:, J] c) and qiht_top_s (H_s) against the CPU oracle on the same seeded inputs.

Tolerances come from the arithmetic:
  gemv_t   r is rounded to 24-bit block fixed point (step 2^(e-22), e the exponent
           with max |r| < 2^e), sums are exact integers, one final rounding:
           |g_j - g*_j| <= alpha sum_i |W_ij| 2^(e-23) + 2^-24 |g*_j|
  gemv_cols  FP32 fused multiply-adds over k terms and the chunk sums:
           |z_i - z*_i| <= 1.1 (2k + 4) 2^-24 alpha sum_j |W_ij c_j|
  top_s    exact: the same binary32 values, compared as indices
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_04907_gb300 as q
import synth

pytestmark = pytest.mark.gpu


def _deq(v, bits, seed, stream):
    codes, c = oracle.quantize(v, bits, seed, stream)
    return oracle.dequantize(codes, bits, c), codes, c


GEMV_SHAPES = [(17, 5), (256, 1024), (1000, 333), (2048, 129), (4512, 640), (8192, 700), (16384, 64)]


@pytest.mark.parametrize("bits", [2, 4, 8])
@pytest.mark.parametrize("shape", GEMV_SHAPES)
def test_gemv_t(bits, shape):
    m, n = shape
    v = synth.random_floats((m, n), seed=m + n)
    r = synth.random_floats(m, seed=m * 3 + 1, scale=0.37)
    r[m // 3] *= 50.0                      # one large entry: wide dynamic range
    Q = q.quantize(torch.from_numpy(v).cuda(), bits, 4, 0)
    g = q.gemv_t(Q, torch.from_numpy(r).cuda()).cpu().numpy().astype(np.float64)
    A, codes, c = _deq(v, bits, 4, 0)
    ref = oracle.gemv_t(A, r.astype(np.float64))
    L = 2**bits
    alpha = c / (L - 1)
    e = np.frexp(np.max(np.abs(r)).astype(np.float64))[1]
    absW = np.abs(2.0 * codes.astype(np.float64) - (L - 1))
    bound = (alpha * absW.sum(axis=0) * 2.0 ** (e - 23) + 2.0**-24 * np.abs(ref)) * (1 + 2.0**-20) + 1e-30
    err = np.abs(g - ref)
    assert np.all(err <= bound), (err / bound).max()


def test_gemv_t_zero_residual():
    v = synth.random_floats((300, 50), seed=1)
    Q = q.quantize(torch.from_numpy(v).cuda(), 8, 4, 0)
    g = q.gemv_t(Q, torch.zeros(300, device="cuda"))
    assert torch.all(g == 0)


@pytest.mark.parametrize("bits", [2, 4, 8])
@pytest.mark.parametrize("shape,count", [((17, 40), 3), ((1000, 500), 77), ((8192, 4096), 512), ((4512, 300), 8)])
def test_gemv_cols(bits, shape, count):
    m, n = shape
    v = synth.random_floats((m, n), seed=n)
    rng = np.random.Generator(np.random.PCG64(count))
    cols = rng.choice(n, count, replace=False).astype(np.int32)
    coef = rng.standard_normal(count).astype(np.float32)
    Q = q.quantize(torch.from_numpy(v).cuda(), bits, 9, 1)
    z = q.gemv_cols(Q, torch.from_numpy(cols).cuda(), torch.from_numpy(coef).cuda()).cpu().numpy()
    A, codes, c = _deq(v, bits, 9, 1)
    ref = oracle.gemv_cols(A, cols, coef.astype(np.float64))
    mag = np.abs(A[:, cols]) @ np.abs(coef.astype(np.float64))
    bound = 1.1 * (2 * count + 4) * 2.0**-24 * mag + 1e-30
    assert np.all(np.abs(z - ref) <= bound), (np.abs(z - ref) / bound).max()


@pytest.mark.parametrize("bad", [-1, 40, 2**31 - 1])
def test_gemv_cols_index_out_of_range_gives_nan(bad):
    # a caller's column index outside [0, cols) is never used to address the codes: the
    # product is marked invalid (every entry of z NaN) instead; the next call is unaffected
    m, n = 300, 40
    v = synth.random_floats((m, n), seed=3)
    Q = q.quantize(torch.from_numpy(v).cuda(), 8, 9, 1)
    cols = torch.tensor([3, bad, 7] + list(range(10, 20)), dtype=torch.int32, device="cuda")
    coef = torch.ones(cols.numel(), dtype=torch.float32, device="cuda")
    z = q.gemv_cols(Q, cols, coef)
    torch.cuda.synchronize()
    assert torch.all(torch.isnan(z))
    good = q.gemv_cols(Q, cols[[0, 2]].contiguous(), coef[:2].contiguous())
    torch.cuda.synchronize()
    assert torch.all(torch.isfinite(good))


@pytest.mark.parametrize("n,s", [(1, 1), (5, 5), (7, 3), (1024, 16), (1000, 999), (32768, 256), (49152, 1000),
                                 (16384, 64), (40000, 1),
                                 # past one CTA's 49152 keys: the multi-CTA radix select
                                 (49153, 100), (262144, 512), (262144, 1), (100000, 99999), (300000, 300000),
                                 (1 << 20, 4096)])
def test_top_s(n, s):
    rng = np.random.Generator(np.random.PCG64(n + s))
    a = rng.standard_normal(n).astype(np.float32)
    a[rng.choice(n, n // 3, replace=False)] = np.round(a[: n // 3], 1)   # ties
    idx, val, kth = q.top_s(torch.from_numpy(a).cuda(), s)
    ref, rkth = oracle.top_s(a.astype(np.float64), s)
    assert np.array_equal(idx.cpu().numpy(), ref)
    assert np.array_equal(val.cpu().numpy(), a[ref])
    assert np.array_equal(kth.cpu().numpy().astype(np.float64), rkth)


def test_top_s_all_equal_and_zeros():
    for a in (np.zeros(1000, np.float32), np.full(777, -2.5, np.float32), np.zeros(70000, np.float32),
              np.full(123457, 3.0, np.float32)):
        idx, _, kth = q.top_s(torch.from_numpy(a).cuda(), 10)
        assert np.array_equal(idx.cpu().numpy(), np.arange(10))
        assert kth[0].item() == abs(a[0]) and kth[1].item() == abs(a[0])


def test_top_s_multi_cta_magnitude_ties_across_chunks():
    # equal magnitudes of both signs spread over many chunks: the lowest indices win
    n, s = 200000, 5000
    a = np.zeros(n, np.float32)
    rng = np.random.Generator(np.random.PCG64(11))
    hot = np.sort(rng.choice(n, 9000, replace=False))
    a[hot] = np.where(rng.random(9000) < 0.5, -1.25, 1.25).astype(np.float32)
    a[hot[:100]] = 2.0                                    # above the tie level
    idx, val, kth = q.top_s(torch.from_numpy(a).cuda(), s)
    ref, rkth = oracle.top_s(a.astype(np.float64), s)
    assert np.array_equal(idx.cpu().numpy(), ref)
    assert np.array_equal(val.cpu().numpy(), a[ref])
    assert np.array_equal(kth.cpu().numpy().astype(np.float64), rkth)


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_gemv_t_full_size_sampled(bits):
    # 8192 x 32768 (the large single-solve workload) at every width, in the launch shape the
    # solver uses: sampled columns against the oracle
    p = synth.large_noisy(seed=0)
    r = synth.random_floats(p.m, seed=77, scale=0.01)
    L = (1 << bits) - 1
    Q = q.quantize(torch.from_numpy(p.phi).cuda(), bits, 5, 0)
    g = q.gemv_t(Q, torch.from_numpy(r).cuda()).cpu().numpy().astype(np.float64)
    c, _ = oracle.absmax(p.phi)
    e = np.frexp(np.max(np.abs(r)).astype(np.float64))[1]
    rng = np.random.Generator(np.random.PCG64(1))
    for j in np.concatenate([[0, p.n - 1], rng.choice(p.n, 30, replace=False)]):
        codes, _ = oracle.quantize(np.ascontiguousarray(p.phi[:, j]), bits, 5, 0, c, col0=int(j), rows_total=p.m)
        col = oracle.dequantize(codes, bits, c)
        ref = float(oracle.gemv_t(col[:, None], r.astype(np.float64))[0])
        bound = ((c / L) * np.abs(2.0 * codes - L).sum() * 2.0 ** (e - 23) + 2.0**-24 * abs(ref)) * (1 + 2.0**-20)
        assert abs(g[j] - ref) <= bound, j


# ---- products on the odd grid (2^(b-1) + 1 levels): the same bounds with L - 1 = 2^(b-1) ----

@pytest.mark.parametrize("bits", [2, 4, 8])
@pytest.mark.parametrize("shape", [(17, 5), (1000, 333), (4512, 640), (16384, 64)])
def test_gemv_t_odd_grid(bits, shape):
    m, n = shape
    v = synth.random_floats((m, n), seed=m + 2 * n)
    r = synth.random_floats(m, seed=m * 5 + 2, scale=0.41)
    r[m // 2] *= 40.0
    Q = q.quantize(torch.from_numpy(v).cuda(), bits, 6, 1, odd=True)
    g = q.gemv_t(Q, torch.from_numpy(r).cuda()).cpu().numpy().astype(np.float64)
    codes, c = oracle.quantize(v, bits, 6, 1, odd=True)
    A = oracle.dequantize(codes, bits, c, odd=True)
    ref = oracle.gemv_t(A, r.astype(np.float64))
    lm1 = 2 ** (bits - 1)
    alpha = c / lm1
    e = np.frexp(np.max(np.abs(r)).astype(np.float64))[1]
    absW = np.abs(2.0 * codes.astype(np.float64) - lm1)
    bound = (alpha * absW.sum(axis=0) * 2.0 ** (e - 23) + 2.0**-24 * np.abs(ref)) * (1 + 2.0**-20) + 1e-30
    err = np.abs(g - ref)
    assert np.all(err <= bound), (err / bound).max()


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_gemv_cols_odd_grid(bits):
    m, n, count = 1000, 500, 77
    v = synth.random_floats((m, n), seed=n + 1)
    rng = np.random.Generator(np.random.PCG64(count + 1))
    cols = rng.choice(n, count, replace=False).astype(np.int32)
    coef = rng.standard_normal(count).astype(np.float32)
    Q = q.quantize(torch.from_numpy(v).cuda(), bits, 9, 1, odd=True)
    z = q.gemv_cols(Q, torch.from_numpy(cols).cuda(), torch.from_numpy(coef).cuda()).cpu().numpy()
    codes, c = oracle.quantize(v, bits, 9, 1, odd=True)
    A = oracle.dequantize(codes, bits, c, odd=True)
    ref = oracle.gemv_cols(A, cols, coef.astype(np.float64))
    mag = np.abs(A[:, cols]) @ np.abs(coef.astype(np.float64))
    bound = 1.1 * (2 * count + 4) * 2.0**-24 * mag + 1e-30
    assert np.all(np.abs(z - ref) <= bound), (np.abs(z - ref) / bound).max()
