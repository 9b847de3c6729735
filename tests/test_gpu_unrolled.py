"""K unrolled QIHT iterations and their adjoint on the GPU (qiht_unrolled_forward/_backward)
against the CPU oracle (oracle/unrolled.py, whose adjoint is pinned by finite differences).

Both sides use the same quantized codes (bit-exact, see test_gpu_quantize.py). Tolerances:
x_K within 1e-4 relative L2 (FP32 products of s columns, FP64 sums), with identical supports;
the gradients within 2e-3 relative L2 (FP32 products in every one of the K adjoint steps and
the recomputed forward). Problems whose selections the oracle finds ambiguous (relative gap
between the s-th and (s+1)-th magnitude below 1e-5) are excluded from the support check."""
import numpy as np
import pytest
import torch

import oracle
from oracle import unrolled
import paper_1802_04907_gb300 as q

pytestmark = pytest.mark.gpu


def _problems(P, m, n, s, bits, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for p in range(P):
        phi = (rng.standard_normal((m, n)) / np.sqrt(m)).astype(np.float32)
        x = np.zeros(n)
        x[rng.choice(n, s, replace=False)] = rng.standard_normal(s)
        mag, ph = rng.uniform(0.9, 1.1, m), rng.uniform(-0.1, 0.1, m)
        a, b = mag * np.cos(ph), mag * np.sin(ph)
        clean = unrolled.stacked(phi.astype(np.float64), a, b) @ x
        y = clean + np.sqrt(clean @ clean / (2 * m * 1e3)) * rng.standard_normal(2 * m)
        out.append((phi, x, a.astype(np.float32), b.astype(np.float32), y.astype(np.float32)))
    return out


def _setup(P, m, n, s, bits, K, seed):
    probs = _problems(P, m, n, s, bits, seed)
    Q1s, Q2s, refs = [], [], []
    for p, (phi, x, a, b, y) in enumerate(probs):
        t = torch.from_numpy(phi).cuda()
        q1, q2 = q.quantize_pair(t, bits, 100 + p, q.STREAM_Q1, q.STREAM_Q2)
        Q1s.append(q1)
        Q2s.append(q2)
        c1, sc = oracle.quantize(phi, bits, 100 + p, 0)
        c2, _ = oracle.quantize(phi, bits, 100 + p, 1, sc)
        refs.append((oracle.dequantize(c1, bits, sc), oracle.dequantize(c2, bits, sc)))
    Y = torch.from_numpy(np.stack([pr[4] for pr in probs])).cuda()
    GA = torch.from_numpy(np.stack([pr[2] for pr in probs])).cuda()
    GB = torch.from_numpy(np.stack([pr[3] for pr in probs])).cuda()
    XT = torch.from_numpy(np.stack([pr[1] for pr in probs]).astype(np.float32)).cuda()
    op = q.Unrolled(Q1s, Q2s, s, K)
    return probs, refs, op, Y, GA, GB, XT


def _min_gap(steps, s):
    g = np.inf
    for st in steps:
        z = np.abs(st.x + st.mu * st.h)
        srt = np.sort(z)[::-1]
        if srt[s - 1] > 0:
            g = min(g, (srt[s - 1] - srt[s]) / srt[s - 1])
    return g


@pytest.mark.parametrize("bits,K,P,m,n,s", [(4, 6, 4, 256, 1024, 12), (8, 12, 4, 256, 1024, 12),
                                            (2, 5, 4, 256, 1024, 12),
                                            # ragged: columns off the 4-column groups, rows off a
                                            # 512-byte batch, problems split across CTAs
                                            (4, 5, 5, 333, 1001, 9), (2, 4, 7, 700, 1003, 11),
                                            (8, 4, 3, 1500, 2047, 16)])
def test_forward_and_adjoint_match_oracle(bits, K, P, m, n, s):
    probs, refs, op, Y, GA, GB, XT = _setup(P, m, n, s, bits, K, seed=bits * 10 + K)
    X = op.forward(Y, GA, GB)
    Xbar = 2.0 * (X - XT)
    yb, ab, bb = op.backward(Y, GA, GB, Xbar)
    torch.cuda.synchronize()
    X, yb, ab, bb = (t.cpu().numpy().astype(np.float64) for t in (X, yb, ab, bb))
    checked = 0
    for p, (phi, x, a, b, y) in enumerate(probs):
        P1, P2 = refs[p]
        xK, steps = unrolled.forward(P1, P2, y, a, b, s, K)
        if _min_gap(steps, s) < 1e-5:
            continue
        checked += 1
        assert np.array_equal(np.flatnonzero(X[p]), np.flatnonzero(xK)), p
        assert np.linalg.norm(X[p] - xK) <= 1e-4 * np.linalg.norm(xK), p
        gy, ga, gb = unrolled.backward(P1, P2, a, b, steps, 2.0 * (xK - x))
        for got, want, name in ((yb[p], gy, "y"), (ab[p], ga, "a"), (bb[p], gb, "b")):
            rel = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30)
            assert rel <= 2e-3, (p, name, rel)
    assert checked >= 2


def test_checkpointed_segments_long_unroll():
    # K = 50: ceil(sqrt(50)) = 8-step segments (the last one short), each recomputed in the adjoint
    P, m, n, s, K = 3, 192, 768, 10, 50
    probs, refs, op, Y, GA, GB, XT = _setup(P, m, n, s, 4, K, seed=77)
    X = op.forward(Y, GA, GB)
    yb, ab, bb = op.backward(Y, GA, GB, 2.0 * (X - XT))
    torch.cuda.synchronize()
    X, yb, ab, bb = (t.cpu().numpy().astype(np.float64) for t in (X, yb, ab, bb))
    checked = 0
    for p, (phi, x, a, b, y) in enumerate(probs):
        P1, P2 = refs[p]
        xK, steps = unrolled.forward(P1, P2, y, a, b, s, K)
        if _min_gap(steps, s) < 1e-5:
            continue
        checked += 1
        assert np.linalg.norm(X[p] - xK) <= 1e-4 * np.linalg.norm(xK), p
        gy, ga, gb = unrolled.backward(P1, P2, a, b, steps, 2.0 * (xK - x))
        for got, want in ((yb[p], gy), (ab[p], ga), (bb[p], gb)):
            assert np.linalg.norm(got - want) <= 5e-3 * np.linalg.norm(want), p
    assert checked >= 1


def test_autograd_function_and_repeat_calls():
    P, m, n, s, K = 2, 128, 512, 8, 7
    probs, refs, op, Y, GA, GB, XT = _setup(P, m, n, s, 8, K, seed=5)
    y = Y.clone().requires_grad_(True)
    ga = GA.clone().requires_grad_(True)
    gb = GB.clone().requires_grad_(True)
    X = q.unrolled_qiht(y, ga, gb, op)
    loss = ((X - XT) ** 2).sum()
    loss.backward()
    X2 = op.forward(Y, GA, GB)
    yb, ab, bb = op.backward(Y, GA, GB, 2.0 * (X2 - XT))
    torch.cuda.synchronize()
    assert torch.equal(X.detach(), X2)
    assert torch.equal(y.grad, yb) and torch.equal(ga.grad, ab) and torch.equal(gb.grad, bb)


def test_full_size_sampled_problems():
    # the differentiation workload at full size, in the launch configuration of the benchmark:
    # 64 problems, Gaussian Phi 2048 x 8192 N(0, 1/m), s = 64, 4-bit codes, per-row complex gain,
    # 30 dB, K = 50 unrolled iterations with sqrt(K) checkpoints; three sampled problems (first,
    # middle, last) against the oracle's forward and adjoint
    P, m, n, s, K, bits = 64, 2048, 8192, 64, 50, 4
    pick = (0, 31, 63)
    rng = np.random.Generator(np.random.PCG64(2048))
    Q1s, Q2s, Y, GA, GB, XT, keep = [], [], [], [], [], [], {}
    for p in range(P):
        phi = rng.standard_normal((m, n), dtype=np.float32) * np.float32(1.0 / np.sqrt(m))
        sup = rng.choice(n, s, replace=False)
        x = np.zeros(n)
        x[sup] = rng.standard_normal(s)
        mag, ph = rng.uniform(0.9, 1.1, m), rng.uniform(-0.1, 0.1, m)
        a, b = (mag * np.cos(ph)).astype(np.float32), (mag * np.sin(ph)).astype(np.float32)
        px = phi[:, sup].astype(np.float64) @ x[sup]
        clean = np.concatenate([a * px, b * px])
        y = (clean + np.sqrt(clean @ clean / (2 * m * 1e3)) * rng.standard_normal(2 * m)).astype(np.float32)
        q1, q2 = q.quantize_pair(torch.from_numpy(phi).cuda(), bits, 100 + p, q.STREAM_Q1, q.STREAM_Q2)
        Q1s.append(q1)
        Q2s.append(q2)
        Y.append(y)
        GA.append(a)
        GB.append(b)
        XT.append(x.astype(np.float32))
        if p in pick:
            keep[p] = (phi, x, a, b, y)
    Yt, GAt, GBt, XTt = (torch.from_numpy(np.stack(v)).cuda() for v in (Y, GA, GB, XT))
    op = q.Unrolled(Q1s, Q2s, s, K)
    X = op.forward(Yt, GAt, GBt)
    yb, ab, bb = op.backward(Yt, GAt, GBt, 2.0 * (X - XTt))
    torch.cuda.synchronize()
    X, yb, ab, bb = (t.cpu().numpy().astype(np.float64) for t in (X, yb, ab, bb))
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(yb)) and np.all(np.isfinite(ab))
    assert all(np.count_nonzero(X[p]) <= s for p in range(P))
    checked = 0
    for p in pick:
        phi, x, a, b, y = keep[p]
        c1, sc = oracle.quantize(phi, bits, 100 + p, 0)
        c2, _ = oracle.quantize(phi, bits, 100 + p, 1, sc)
        P1, P2 = oracle.dequantize(c1, bits, sc), oracle.dequantize(c2, bits, sc)
        xK, steps = unrolled.forward(P1, P2, y, a, b, s, K)
        if _min_gap(steps, s) < 1e-5:
            continue
        checked += 1
        assert np.array_equal(np.flatnonzero(X[p]), np.flatnonzero(xK)), p
        assert np.linalg.norm(X[p] - xK) <= 1e-4 * np.linalg.norm(xK), p
        gy, ga, gb = unrolled.backward(P1, P2, a, b, steps, 2.0 * (xK - x))
        for got, want, name in ((yb[p], gy, "y"), (ab[p], ga, "a"), (bb[p], gb, "b")):
            rel = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30)
            assert rel <= 5e-3, (p, name, rel)
    assert checked >= 2


def test_zero_iterations_give_zero_output_and_gradients():
    P, m, n, s = 2, 64, 200, 5
    probs, refs, op, Y, GA, GB, XT = _setup(P, m, n, s, 8, 0, seed=3)
    X = op.forward(Y, GA, GB)
    yb, ab, bb = op.backward(Y, GA, GB, 2.0 * (X - XT))
    torch.cuda.synchronize()
    assert torch.all(X == 0)
    assert torch.all(yb == 0) and torch.all(ab == 0) and torch.all(bb == 0)


@pytest.mark.parametrize("bits,K,P,m,n,s", [(8, 1, 3, 40, 37, 1),      # one step, s = 1, n off every tile
                                            (4, 2, 2, 16, 64, 16),     # s = m
                                            (2, 3, 2, 33, 129, 7)])
def test_edge_shapes_against_oracle(bits, K, P, m, n, s):
    probs, refs, op, Y, GA, GB, XT = _setup(P, m, n, s, bits, K, seed=bits + 7 * K + m)
    X = op.forward(Y, GA, GB)
    yb, ab, bb = op.backward(Y, GA, GB, 2.0 * (X - XT))
    torch.cuda.synchronize()
    X, yb, ab, bb = (t.cpu().numpy().astype(np.float64) for t in (X, yb, ab, bb))
    checked = 0
    for p, (phi, x, a, b, y) in enumerate(probs):
        P1, P2 = refs[p]
        xK, steps = unrolled.forward(P1, P2, y, a, b, s, K)
        assert np.count_nonzero(X[p]) <= s
        if s < n and _min_gap(steps, s) < 1e-5:
            continue
        checked += 1
        assert np.array_equal(np.flatnonzero(X[p]), np.flatnonzero(xK)), p
        assert np.linalg.norm(X[p] - xK) <= 1e-4 * max(np.linalg.norm(xK), 1e-30), p
        gy, ga, gb = unrolled.backward(P1, P2, a, b, steps, 2.0 * (xK - x))
        for got, want, name in ((yb[p], gy, "y"), (ab[p], ga, "a"), (bb[p], gb, "b")):
            rel = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30)
            assert rel <= 2e-3, (p, name, rel)
    assert checked >= 1
