"""Many right-hand sides sharing one quantized matrix.

qiht_gemv_t_multi (G = Q^T R on the tensor cores) against the CPU oracle's FP64
product of the dequantized codes. Tolerance from the arithmetic: the centred codes are
exact in f16; each residual is scaled by a power of two and split into f16 parts
hi + lo with |r' - hi - lo| <= 2^-22 |r'| + 2^-25 (r' <= 2^15); products are exact;
the K = rows products are summed in FP32, at most one rounding per 16-term MMA step
and per accumulation (bounded here by 2 (K/16 + 2) 2^-24 of the sum of magnitudes);
one final scaling by alpha 2^e (two roundings). With S = alpha sum_i |W_ij r_i|:
  |G - G*| <= (2 (K/16 + 2) 2^-24 + 2^-21) S + 2^-22 |G*|
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_04907_gb300 as q
import synth

pytestmark = pytest.mark.gpu


def _multi_bound(codes, lm1, c, R, ref):
    W = np.abs(2.0 * codes.astype(np.float64) - lm1)          # m x n
    S = (c / lm1) * (np.abs(R.astype(np.float64)) @ W)       # nrhs x n
    K = codes.shape[0]
    return (2 * (np.ceil(K / 16) + 2) * 2.0**-24 + 2.0**-21) * S + 2.0**-22 * np.abs(ref) + 1e-30


@pytest.mark.parametrize("bits", [2, 4, 8])
@pytest.mark.parametrize("m,n,nrhs", [(17, 5, 3), (1000, 333, 37), (4512, 640, 300), (8192, 256, 256)])
def test_gemv_t_multi(bits, m, n, nrhs):
    v = synth.random_floats((m, n), seed=m + n + bits)
    R = synth.random_floats((nrhs, m), seed=m * 7 + nrhs, scale=0.3)
    R[:, m // 3] *= 50.0                                      # wide dynamic range
    R[nrhs // 2, :] = 0.0                                     # a zero residual
    Q = q.quantize(torch.from_numpy(v).cuda(), bits, 4, 0)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    G = q.gemv_t_multi(Q, torch.from_numpy(R).cuda(), status=status).cpu().numpy().astype(np.float64)
    assert status.item() == q.OK
    codes, c = oracle.quantize(v, bits, 4, 0)
    A = oracle.dequantize(codes, bits, c)
    ref = np.stack([oracle.gemv_t(A, R[k].astype(np.float64)) for k in range(nrhs)])
    bound = _multi_bound(codes, 2**bits - 1, c, R, ref)
    err = np.abs(G - ref)
    ratio = (err / bound).max()
    print(f"bits={bits} m={m} n={n} nrhs={nrhs}: max err/bound {ratio:.3e}")
    assert np.all(err <= bound), ratio
    assert np.all(G[nrhs // 2] == 0.0)


def test_gemv_t_multi_matches_single_products():
    # the same residuals through the exact integer GEMV^T one by one
    m, n, nrhs = 2048, 1000, 40
    v = synth.random_floats((m, n), seed=3)
    R = synth.random_floats((nrhs, m), seed=4)
    Q = q.quantize(torch.from_numpy(v).cuda(), 8, 1, 0)
    Rg = torch.from_numpy(R).cuda()
    G = q.gemv_t_multi(Q, Rg).cpu().numpy().astype(np.float64)
    single = np.stack([q.gemv_t(Q, Rg[k].contiguous()).cpu().numpy().astype(np.float64) for k in range(nrhs)])
    scale = np.abs(single).max(axis=1, keepdims=True)
    assert np.all(np.abs(G - single) <= 1e-5 * scale), (np.abs(G - single) / scale).max()


def test_gemv_t_multi_odd_grid():
    m, n, nrhs = 3000, 700, 70
    v = synth.random_floats((m, n), seed=5)
    R = synth.random_floats((nrhs, m), seed=6)
    Q = q.quantize(torch.from_numpy(v).cuda(), 4, 2, 1, odd=True)
    G = q.gemv_t_multi(Q, torch.from_numpy(R).cuda()).cpu().numpy().astype(np.float64)
    codes, c = oracle.quantize(v, 4, 2, 1, odd=True)
    A = oracle.dequantize(codes, 4, c, odd=True)
    ref = np.stack([oracle.gemv_t(A, R[k].astype(np.float64)) for k in range(nrhs)])
    bound = _multi_bound(codes, 2**3, c, R, ref)
    assert np.all(np.abs(G - ref) <= bound)
