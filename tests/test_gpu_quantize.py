"""GPU quantizer (qiht_quantize) vs the CPU oracle: codes bit-exact, scales exact.

Shapes span several 128 x 32 tiles with ragged tails (rows not a multiple of
the codes per word, columns not a multiple of 32), vectors, strided inputs,
a zero matrix, non-finite inputs, and the full-size 8192 x 32768 matrix on
sampled columns."""
import numpy as np
import pytest
import torch

import layout
import oracle
import paper_1802_04907_gb300 as q
import synth

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (3, 5), (37, 53), (128, 33), (257, 100), (1000, 7), (4512, 64), (129, 1)]


@pytest.mark.parametrize("bits", [2, 4, 8])
@pytest.mark.parametrize("shape", SHAPES)
def test_codes_bit_exact(bits, shape):
    m, n = shape
    v = synth.random_floats((m, n), seed=m * 7 + n + bits)
    seed = 0xDEADBEEF12345 + bits
    Q = q.quantize(torch.from_numpy(v).cuda(), bits, seed, 1)
    torch.cuda.synchronize()
    want, c = oracle.quantize(v, bits, seed, 1)
    assert Q.scale.item() == c
    words = Q.words.cpu().numpy()
    assert np.array_equal(layout.unpack(words, m, n, bits), want)
    assert layout.padding_is_zero(words, m, n, bits)


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_vector_and_given_scale(bits):
    m, n = 1001, 17
    v = synth.random_floats((m, n), seed=5)
    y = synth.random_floats(m, seed=6)
    phi = torch.from_numpy(v).cuda()
    q1, q2, qy = q.quantize_problem(phi, torch.from_numpy(y).cuda(), bits, bits, seed=99)
    torch.cuda.synchronize()
    c1, c = oracle.quantize(v, bits, 99, 0)
    c2, _ = oracle.quantize(v, bits, 99, 1, c)
    cy, sy = oracle.quantize(y, bits, 99, 2)
    assert np.array_equal(layout.unpack(q1.words.cpu().numpy(), m, n, bits), c1)
    assert np.array_equal(layout.unpack(q2.words.cpu().numpy(), m, n, bits), c2)
    assert np.array_equal(layout.unpack(qy.words.cpu().numpy(), m, 1, bits)[:, 0], cy)
    assert qy.scale.item() == sy and q2.scale.item() == c


def test_strided_input():
    big = synth.random_floats((300, 90), seed=2)
    t = torch.from_numpy(big).cuda()[:, 10:73]
    assert t.stride(0) == 90
    Q = q.quantize(t, 4, 7, 0)
    torch.cuda.synchronize()
    want, c = oracle.quantize(np.ascontiguousarray(big[:, 10:73]), 4, 7, 0)
    assert Q.scale.item() == c
    assert np.array_equal(layout.unpack(Q.words.cpu().numpy(), 300, 63, 4), want)


def test_zero_matrix():
    v = np.zeros((64, 40), dtype=np.float32)
    Q = q.quantize(torch.from_numpy(v).cuda(), 8, 1, 0)
    torch.cuda.synchronize()
    want, c = oracle.quantize(v, 8, 1, 0)
    assert Q.scale.item() == 0.0 and c == 0.0
    assert np.array_equal(layout.unpack(Q.words.cpu().numpy(), 64, 40, 8), want)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_is_reported(bad):
    v = synth.random_floats((50, 20), seed=1)
    v[13, 7] = bad
    with pytest.raises(q.QihtError) as e:
        q.quantize(torch.from_numpy(v).cuda(), 8, 1, 0, check_finite=True)
    assert e.value.status == q.ERR_NONFINITE


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_full_size_sampled_columns(bits):
    # 8192 x 32768 (the large single-solve workload), sampled columns checked exactly
    p = synth.large_noisy(seed=0)
    phi = torch.from_numpy(p.phi).cuda()
    Q = q.quantize(phi, bits, 12345, 0)
    torch.cuda.synchronize()
    c, bad = oracle.absmax(p.phi)
    assert bad == 0 and Q.scale.item() == c
    rng = np.random.Generator(np.random.PCG64(bits))
    cols = np.concatenate([[0, 31, 32, p.n - 1], rng.choice(p.n, 12, replace=False)])
    ldw = q.ld_words(p.m, bits)
    words = Q.words.view(p.n, ldw)
    for j in cols:
        want, _ = oracle.quantize(np.ascontiguousarray(p.phi[:, j]), bits, 12345, 0, c, col0=int(j), rows_total=p.m)
        got = layout.unpack(words[j].cpu().numpy(), p.m, 1, bits)[:, 0]
        assert np.array_equal(got, want), j


@pytest.mark.parametrize("bits", [2, 4, 8])
@pytest.mark.parametrize("shape", SHAPES)
def test_pair_equals_two_single_quantizations(bits, shape):
    # qiht_quantize_pair (Q1 and Q2 in one pass) is element by element the two single calls
    m, n = shape
    v = torch.from_numpy(synth.random_floats((m, n), seed=m + 3 * n + bits)).cuda()
    qa, qb = q.quantize_pair(v, bits, 1234567, 0, 1)
    sa = q.quantize(v, bits, 1234567, 0)
    sb = q.quantize(v, bits, 1234567, 1, scale=sa.scale.clone(), scale_given=True)
    torch.cuda.synchronize()
    assert qa.scale.item() == sa.scale.item()
    assert torch.equal(qa.words, sa.words) and torch.equal(qb.words, sb.words)
    assert not torch.equal(qa.words, qb.words) or m * n < 4


@pytest.mark.parametrize("offset,ld", [(8, 96), (10, 90), (0, 64)])
def test_pair_strided_input(offset, ld):
    # aligned strides take the float4 path, odd ones the element path; ragged last columns
    big = synth.random_floats((301, ld), seed=offset + ld)
    cols = min(57, ld - offset)
    t = torch.from_numpy(big).cuda()[:, offset:offset + cols]
    qa, qb = q.quantize_pair(t, 8, 77, 0, 1)
    torch.cuda.synchronize()
    sub = np.ascontiguousarray(big[:, offset:offset + cols])
    wa, c = oracle.quantize(sub, 8, 77, 0)
    wb, _ = oracle.quantize(sub, 8, 77, 1, c)
    assert qa.scale.item() == c
    assert np.array_equal(layout.unpack(qa.words.cpu().numpy(), 301, cols, 8), wa)
    assert np.array_equal(layout.unpack(qb.words.cpu().numpy(), 301, cols, 8), wb)


# ---- the odd grid (2^(b-1) + 1 levels, the Appendix's remark on fixed-point hardware) ----

@pytest.mark.parametrize("bits", [2, 4, 8])
@pytest.mark.parametrize("shape", [(3, 5), (257, 100), (4512, 64), (129, 1)])
def test_odd_grid_codes_bit_exact(bits, shape):
    m, n = shape
    v = synth.random_floats((m, n), seed=m * 3 + n + bits)
    v[m // 2, :] = 0.0                      # zeros land on the zero level
    seed = 0x5EED0DD + bits
    Q = q.quantize(torch.from_numpy(v).cuda(), bits, seed, 2, odd=True)
    torch.cuda.synchronize()
    want, c = oracle.quantize(v, bits, seed, 2, odd=True)
    assert Q.scale.item() == c and Q.levels == q.odd_levels(bits) and Q.odd
    words = Q.words.cpu().numpy()
    got = layout.unpack(words, m, n, bits)
    assert np.array_equal(got, want)
    assert got.max() <= 2 ** (bits - 1)
    if c > 0:
        assert np.all(got[m // 2, :] == 2 ** (bits - 2))
    assert layout.padding_is_zero(words, m, n, bits)


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_odd_grid_problem_quantization(bits):
    m, n = 1001, 77
    v = synth.random_floats((m, n), seed=15)
    y = synth.random_floats(m, seed=16)
    q1, q2, qy = q.quantize_problem(torch.from_numpy(v).cuda(), torch.from_numpy(y).cuda(), bits, bits, seed=3,
                                    odd=True)
    torch.cuda.synchronize()
    c1, c = oracle.quantize(v, bits, 3, 0, odd=True)
    c2, _ = oracle.quantize(v, bits, 3, 1, c, odd=True)
    cy, sy = oracle.quantize(y, bits, 3, 2, odd=True)
    assert np.array_equal(layout.unpack(q1.words.cpu().numpy(), m, n, bits), c1)
    assert np.array_equal(layout.unpack(q2.words.cpu().numpy(), m, n, bits), c2)
    assert np.array_equal(layout.unpack(qy.words.cpu().numpy(), m, 1, bits)[:, 0], cy)
    assert q1.levels == q2.levels == qy.levels == q.odd_levels(bits)
    assert qy.scale.item() == sy and q1.scale.item() == c
