"""Phi computed on the fly (qiht_fly_quantize, qiht_gemv_t_fly, qiht_niht_solve_fresh_fly) for the
gridded interferometry matrix, against the CPU oracle on the materialized matrix.

- codes: bit-exact against the oracle's quantizer of the materialized Phi (2/4/8 bits, the odd
  grid, two streams in one pass), scale exact, column padding zero;
- the fused product: within the GEMV^T fixed-point bound of the oracle's FP64 product of the
  dequantized codes, and bitwise equal to qiht_gemv_t on the operator's codes (the same exact
  integer sums and final scaling);
- the fresh-realization solve with Phi from the operator: the parity rule of every solve
  against the oracle's qiht_fresh on the materialized Phi, and bitwise equal to
  qiht_niht_solve_fresh on that matrix.
"""
import numpy as np
import pytest
import torch

import layout
import oracle
import paper_1802_04907_gb300 as q
import synth
from test_gpu_solve import _check

pytestmark = pytest.mark.gpu


def _op(p):
    uv = torch.from_numpy(np.ascontiguousarray(p.meta["uv"], dtype=np.int32)).cuda()
    table = torch.from_numpy(p.meta["table"]).cuda()
    return q.FlyOp(uv, table, p.meta["grid"])


SMALL = [(8, 16), (20, 32), (12, 8)]          # (antennas, grid): K = 56, 380, 132


@pytest.mark.parametrize("bits", [2, 4, 8])
@pytest.mark.parametrize("ant_grid", SMALL)
def test_fly_codes_bit_exact(bits, ant_grid):
    p = synth.interferometry_gridded(ant_grid[0], ant_grid[1], n_src=4, s=4, seed=bits + ant_grid[0])
    op = _op(p)
    seed = 0xC0FFEE + bits
    qa, qb = q.fly_quantize(op, bits, seed, 0, 1)
    torch.cuda.synchronize()
    m, n = p.m, p.n
    for Q, stream in ((qa, 0), (qb, 1)):
        want, c = oracle.quantize(p.phi, bits, seed, stream)
        assert Q.scale.item() == c == 1.0
        words = Q.words.cpu().numpy()
        assert np.array_equal(layout.unpack(words, m, n, bits), want)
        assert layout.padding_is_zero(words, m, n, bits)
    # one quantization alone gives the same words as the first of the pair
    q1 = q.fly_quantize(op, bits, seed, 0)
    assert torch.equal(q1.words, qa.words)


@pytest.mark.parametrize("bits", [4, 8])
def test_fly_codes_odd_grid(bits):
    p = synth.interferometry_gridded(20, 32, n_src=4, s=4, seed=3)
    Q = q.fly_quantize(_op(p), bits, 77, 5, odd=True)
    want, _ = oracle.quantize(p.phi, bits, 77, 5, odd=True)
    assert np.array_equal(layout.unpack(Q.words.cpu().numpy(), p.m, p.n, bits), want)


def test_fly_codes_full_size_sampled():
    # the benchmark's operator: 48 antennas (K = 2256 baselines, 4512 rows), 128 x 128 sky
    p = synth.interferometry_gridded(seed=0)
    Q = q.fly_quantize(_op(p), 8, 11, 0)
    words = Q.words.cpu().numpy().reshape(p.n, -1)
    rng = np.random.Generator(np.random.PCG64(2))
    for j in np.concatenate([[0, p.n // 2 + 64, p.n - 1], rng.choice(p.n, 12, replace=False)]):
        want, _ = oracle.quantize(np.ascontiguousarray(p.phi[:, j]), 8, 11, 0, 1.0, col0=int(j), rows_total=p.m)
        got = layout.unpack(words[j], p.m, 1, 8)[:, 0]
        assert np.array_equal(got, want[:, 0] if want.ndim == 2 else want), j


def _gemv_bound(codes, bits, c, r, ref, L=None):
    L = L or 2**bits
    alpha = c / (L - 1)
    e = np.frexp(np.max(np.abs(r)).astype(np.float64))[1]
    absW = np.abs(2.0 * codes.astype(np.float64) - (L - 1))
    return (alpha * absW.sum(axis=0) * 2.0 ** (e - 23) + 2.0**-24 * np.abs(ref)) * (1 + 2.0**-20) + 1e-30


@pytest.mark.parametrize("bits", [2, 4, 8])
@pytest.mark.parametrize("ant_grid", SMALL + [(48, 128), (66, 16)])   # 66 antennas: 4288 baselines
def test_fly_gemv_t(bits, ant_grid):
    p = synth.interferometry_gridded(ant_grid[0], ant_grid[1], n_src=4, s=4, seed=bits)
    op = _op(p)
    r = synth.random_floats(p.m, seed=p.m + bits, scale=0.4)
    r[p.m // 3] *= 40.0                      # wide dynamic range
    rg = torch.from_numpy(r).cuda()
    g = q.gemv_t_fly(op, bits, 21, 1, rg)
    Q = q.fly_quantize(op, bits, 21, 1)
    g_stored = q.gemv_t(Q, rg)
    torch.cuda.synchronize()
    assert torch.equal(g, g_stored)
    codes, c = oracle.quantize(p.phi, bits, 21, 1)
    ref = oracle.gemv_t(oracle.dequantize(codes, bits, c), r.astype(np.float64))
    err = np.abs(g.cpu().numpy().astype(np.float64) - ref)
    bound = _gemv_bound(codes, bits, c, r, ref)
    assert np.all(err <= bound), (err / bound).max()


def test_fly_gemv_t_odd_grid_and_zero_residual():
    p = synth.interferometry_gridded(20, 32, n_src=4, s=4, seed=9)
    op = _op(p)
    r = synth.random_floats(p.m, seed=4)
    g = q.gemv_t_fly(op, 4, 3, 2, torch.from_numpy(r).cuda(), odd=True)
    codes, c = oracle.quantize(p.phi, 4, 3, 2, odd=True)
    ref = oracle.gemv_t(oracle.dequantize(codes, 4, c, odd=True), r.astype(np.float64))
    bound = _gemv_bound(codes, 4, c, r, ref, L=q.odd_levels(4))
    assert np.all(np.abs(g.cpu().numpy() - ref) <= bound)
    z = q.gemv_t_fly(op, 8, 3, 2, torch.zeros(p.m, device="cuda"))
    assert torch.count_nonzero(z).item() == 0


@pytest.mark.parametrize("bits_phi,bits_y", [(8, 8), (2, 8)])
def test_fresh_fly_against_oracle(bits_phi, bits_y):
    # 20 antennas (380 baselines, 760 rows), 32 x 32 sky, 12 sources, 20 dB, 25 iterations
    p = synth.interferometry_gridded(20, 32, n_src=12, s=12, snr_db=20.0, seed=5)
    y = torch.from_numpy(p.y).cuda()
    sv = q.niht_solve_fresh_fly(_op(p), y, bits_phi, bits_y, 13, p.s, 25, trace=True)
    torch.cuda.synchronize()
    ref, _ = oracle.qiht_fresh(p.phi, p.y, p.s, 25, bits_phi=bits_phi, bits_y=bits_y, seed=13, trace=True)
    _check(sv, ref, p, f"fresh-fly-{bits_phi}/{bits_y}")
    # the same solve from the stored FP32 matrix: identical results
    st = q.niht_solve_fresh(torch.from_numpy(p.phi).cuda(), y, bits_phi, bits_y, 13, p.s, 25, trace=True)
    torch.cuda.synchronize()
    assert torch.equal(sv.x, st.x) and torch.equal(sv.support, st.support)
    assert sv.read_report() == st.read_report()
