"""Many right-hand sides sharing one quantized matrix.

qiht_gemv_t_multi (G = Q^T R on the tensor cores) against the CPU oracle's FP64
product of the dequantized codes. Tolerance from the arithmetic: the centred codes are
exact in f16; each residual is scaled by a power of two and split into f16 parts
hi + lo with |r' - hi - lo| <= 2^-22 |r'| + 2^-25 (r' <= 2^15); products are exact;
the K = rows products are summed in FP32, at most one rounding per 16-term MMA step
and per accumulation (bounded here by 2 (K/16 + 2) 2^-24 of the sum of magnitudes);
one final scaling by alpha 2^e (two roundings). With S = alpha sum_i |W_ij r_i|:
  |G - G*| <= (2 (K/16 + 2) 2^-24 + 2^-21) S + 2^-22 |G*|
The FP8 variant (codes of at most 4 bits, exact in e4m3) holds each residual as three e4m3
terms of r' = r 2^-e (max |r'| in [2^7, 2^8)), |r' - t1 - t2 - t3| <= 2^-12 |r'| + 2^-10, and
sums K/32-term MMA steps in FP32; its solves are compared with the oracle's e4m3 mode, which
forms every gradient from the same three-term residual.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_04907_gb300 as q
import parity
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


@pytest.mark.parametrize("bits,fp8", [(8, False), (4, True)])
def test_gemv_t_multi_full_size_sampled(bits, fp8):
    # the product of the many-right-hand-side workload at full size, in the launch the solver makes
    # every iteration: Q1 of the 8192 x 32768 matrix (8-bit f16 split; 4-bit e4m3 terms) against
    # 1024 residuals; sampled columns of G against the oracle for every right-hand side
    p = synth.large_noisy(seed=0)
    nrhs = 1024
    R = synth.random_floats((nrhs, p.m), seed=91, scale=0.05)
    R[:, p.m // 5] *= 40.0                                    # wide dynamic range
    Q = q.quantize(torch.from_numpy(p.phi).cuda(), bits, 5, 0)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    G = q.gemv_t_multi(Q, torch.from_numpy(R).cuda(), status=status, fp8=fp8).cpu().numpy().astype(np.float64)
    assert status.item() == q.OK and G.shape == (nrhs, p.n)
    c, _ = oracle.absmax(p.phi)
    rng = np.random.Generator(np.random.PCG64(5))
    R64 = R.astype(np.float64)
    lm1 = 2**bits - 1
    for j in np.concatenate([[0, 255, 256, p.n - 1], rng.choice(p.n, 16, replace=False)]):
        codes, _ = oracle.quantize(np.ascontiguousarray(p.phi[:, j]), bits, 5, 0, c, col0=int(j), rows_total=p.m)
        col = oracle.dequantize(codes, bits, c)
        ref = (R64 @ col)[:, None]                            # nrhs x 1
        bound = (_fp8_bound if fp8 else _multi_bound)(codes[:, None], lm1, c, R, ref)
        err = np.abs(G[:, j:j + 1] - ref)
        assert np.all(err <= bound), (j, (err / bound).max())


def _fp8_bound(codes, lm1, c, R, ref):
    """FP8 variant: the residual r' = r 2^-e (max |r'| in [2^7, 2^8)) is three e4m3 terms with
    |r' - t1 - t2 - t3| <= 2^-12 |r'| + 2^-10; the products are exact; FP32 sums over K/32-term
    MMA steps (at most one rounding per step and per accumulation)."""
    W = np.abs(2.0 * codes.astype(np.float64) - lm1)          # m x n
    Ra = np.abs(R.astype(np.float64))
    e = np.frexp(Ra.max(axis=1))[1] - 8                       # per right-hand side
    S = (c / lm1) * (Ra @ W)
    floor = (c / lm1) * (2.0 ** (e - 10))[:, None] * W.sum(axis=0)[None, :]
    K = codes.shape[0]
    return (2.0**-12 + 2 * (np.ceil(K / 32) + 2) * 2.0**-24 + 2.0**-21) * S + floor + 2.0**-22 * np.abs(ref) + 1e-30


@pytest.mark.parametrize("bits", [2, 4])
@pytest.mark.parametrize("m,n,nrhs", [(17, 5, 3), (1000, 333, 37), (4512, 640, 300), (8192, 256, 256)])
def test_gemv_t_multi_fp8(bits, m, n, nrhs):
    # codes of at most 4 bits are exact in e4m3; the residual as three e4m3 terms
    v = synth.random_floats((m, n), seed=m + n + bits)
    R = synth.random_floats((nrhs, m), seed=m * 7 + nrhs, scale=0.3)
    R[:, m // 3] *= 50.0                                      # wide dynamic range
    R[nrhs // 2, :] = 0.0                                     # a zero residual
    Q = q.quantize(torch.from_numpy(v).cuda(), bits, 4, 0)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    G = q.gemv_t_multi(Q, torch.from_numpy(R).cuda(), status=status, fp8=True).cpu().numpy().astype(np.float64)
    assert status.item() == q.OK
    codes, c = oracle.quantize(v, bits, 4, 0)
    A = oracle.dequantize(codes, bits, c)
    ref = np.stack([oracle.gemv_t(A, R[k].astype(np.float64)) for k in range(nrhs)])
    bound = _fp8_bound(codes, 2**bits - 1, c, R, ref)
    err = np.abs(G - ref)
    ratio = (err / bound).max()
    print(f"fp8 bits={bits} m={m} n={n} nrhs={nrhs}: max err/bound {ratio:.3e}")
    assert np.all(err <= bound), ratio
    assert np.all(G[nrhs // 2] == 0.0)


def test_gemv_t_multi_fp8_odd_grid():
    m, n, nrhs = 3000, 700, 70
    v = synth.random_floats((m, n), seed=5)
    R = synth.random_floats((nrhs, m), seed=6)
    Q = q.quantize(torch.from_numpy(v).cuda(), 4, 2, 1, odd=True)
    G = q.gemv_t_multi(Q, torch.from_numpy(R).cuda(), fp8=True).cpu().numpy().astype(np.float64)
    codes, c = oracle.quantize(v, 4, 2, 1, odd=True)
    A = oracle.dequantize(codes, 4, c, odd=True)
    ref = np.stack([oracle.gemv_t(A, R[k].astype(np.float64)) for k in range(nrhs)])
    assert np.all(np.abs(G - ref) <= _fp8_bound(codes, 2**3, c, R, ref))


@pytest.mark.parametrize("bits", [2, 4])
def test_multi_fp8_solve_against_oracle(bits):
    # the many-right-hand-side solve with the FP8 gradient (QIHT_SOLVE_FP8) against the oracle's
    # e4m3 mode (every gradient formed from the residual held as three e4m3 terms), on the
    # strict branch: supports, iteration count, residual and x per right-hand side. The GPU
    # splits its FP32 residual, the oracle its FP64 one; where the two straddle a rounding
    # boundary of the third term (about m/5000 entries an iteration) an entry moves by 2^-11
    # of itself, which moves a gradient entry by about 1e-5 of its size: selections with a
    # relative gap below 1e-4 count as ambiguous here
    s = 8 if bits == 2 else 20
    mp = synth.multi_gaussian(512, 2048, s, 24, seed=bits + 40, snr_db=30.0, values="pm_u")
    res, _ = _multi_run(mp, bits, bits, 40, seed=9, fp8=True)
    # At 2 bits the initial gradient Q1^T Q(y) is an integer combination of few values, and
    # exact ties in its selection are common (about half of these problems); the e4m3 terms
    # split such a tie by rounding only. A fallback at iteration 0 is accepted only where the
    # exact gradient itself ties; later fallbacks are bounded by an eighth.
    late = 0
    for k in range(mp.Y.shape[0]):
        p = mp.problem(k)
        ref, _ = oracle.qiht(p.phi, p.y, s, 40, bits_phi=bits, bits_y=bits, seed=9, trace=True, grad_e4m3=True)
        rep = res.report(k)
        sup = res.support[k].cpu().numpy()
        assert np.all(np.diff(sup) > 0)
        rec = parity.check(f"multi-fp8-{bits}bit[{k}]", ref, mp.X_true[k], x=res.x[k].cpu().numpy(), support=sup,
                           status=rep.status, iters_run=rep.iters_run, resid_norm2=rep.resid_norm2, gap=1e-4)
        if rec["branch"] == "fallback" and rec["first_ambiguous"] == 0:
            ex, _ = oracle.qiht(p.phi, p.y, s, 0, bits_phi=bits, bits_y=bits, seed=9, trace=True)
            assert ex.trace["min_gap"][0] < 1e-12, f"rhs {k}: fallback at iteration 0 without an exact tie"
        elif rec["branch"] == "fallback":
            late += 1
    assert late <= mp.Y.shape[0] // 8


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


# ---- the solver for many right-hand sides (qiht_niht_solve_multi) ----

def _multi_run(mp, bits_phi, bits_y, iters, seed, odd=False, **kw):
    phi = torch.from_numpy(mp.phi).cuda()
    q1, q2 = q.quantize_pair(phi, bits_phi, seed, q.STREAM_Q1, q.STREAM_Q2, odd=odd)
    ys = [q.quantize(torch.from_numpy(mp.Y[k]).cuda(), bits_y, seed, q.STREAM_Y, odd=odd)
          for k in range(mp.Y.shape[0])]
    res = q.niht_solve_multi(q1, q2, ys, mp.s, iters, **kw)
    torch.cuda.synchronize()
    return res, (q1, q2, ys)


def _check_rhs(res, mp, k, ref, tol=1e-4, label="multi"):
    """parity.check for right-hand side k; True when it took the fallback branch."""
    rep = res.report(k)
    sup = res.support[k].cpu().numpy()
    assert np.all(np.diff(sup) > 0)
    rec = parity.check(f"{label}[{k}]", ref, mp.X_true[k], x=res.x[k].cpu().numpy(), support=sup,
                       status=rep.status, iters_run=rep.iters_run, resid_norm2=rep.resid_norm2, x_tol=tol)
    return rec["branch"] == "fallback"


@pytest.mark.parametrize("bits", [2, 4, 8])
def test_multi_against_oracle(bits):
    # 24 observations of one 512 x 2048 Gaussian matrix, s = 20 (8 at 2 bits), 30 dB
    s = 8 if bits == 2 else 20
    mp = synth.multi_gaussian(512, 2048, s, 24, seed=bits, snr_db=30.0, values="pm_u")
    res, _ = _multi_run(mp, bits, bits, 40, seed=9)
    amb = 0
    for k in range(mp.Y.shape[0]):
        p = mp.problem(k)
        ref, _ = oracle.qiht(p.phi, p.y, s, 40, bits_phi=bits, bits_y=bits, seed=9, trace=True)
        amb += _check_rhs(res, mp, k, ref, label=f"multi-{bits}bit")
    # the fallback branch is taken only where the oracle itself is ambiguous; at 2 bits the
    # initial gradient Q1^T Q(y) is a small integer combination of codes times one scale, so
    # exact ties in the initial selection are common there
    assert amb <= mp.Y.shape[0] // (4 if bits == 2 else 8)


def test_multi_ragged_two_tiles_mixed_widths():
    # 300 right-hand sides (two N tiles, the second ragged), m and n off every tile size,
    # 4-bit Phi with 8-bit observations; a sample of them against the oracle
    mp = synth.multi_gaussian(1000, 3001, 15, 300, seed=5, snr_db=25.0, values="normal")
    res, _ = _multi_run(mp, 4, 8, 30, seed=2)
    reps = res.all_reports()
    assert all(r.status == q.OK for r in reps)
    for k in (0, 1, 137, 255, 256, 299):
        p = mp.problem(k)
        ref, _ = oracle.qiht(p.phi, p.y, mp.s, 30, bits_phi=4, bits_y=8, seed=2, trace=True)
        _check_rhs(res, mp, k, ref)


def test_multi_matches_single_solves():
    # the same observations through qiht_niht_solve one by one: same supports, x close
    mp = synth.multi_gaussian(768, 4096, 24, 16, seed=11, snr_db=30.0, values="pm_u")
    res, (q1, q2, ys) = _multi_run(mp, 8, 8, 50, seed=4)
    for k in range(16):
        sv = q.niht_solve(q1, q2, ys[k], mp.s, 50)
        torch.cuda.synchronize()
        rs, rm = sv.read_report(), res.report(k)
        assert rs.status == rm.status == q.OK and rs.iters_run == rm.iters_run, (k, rs, rm)
        assert torch.equal(torch.sort(sv.support).values, res.support[k]), k
        xs, xm = sv.x.double(), res.x[k].double()
        assert (torch.linalg.norm(xs - xm) / torch.linalg.norm(xs)).item() <= 1e-4, k


def test_multi_odd_grid_and_equal_magnitudes():
    mp = synth.multi_gaussian(512, 2048, 16, 12, seed=21, snr_db=30.0, values="ones")
    res, _ = _multi_run(mp, 8, 8, 40, seed=6, odd=True)
    for k in range(12):
        p = mp.problem(k)
        ref, _ = oracle.qiht(p.phi, p.y, mp.s, 40, bits_phi=8, bits_y=8, seed=6, trace=True, odd=True)
        _check_rhs(res, mp, k, ref)


def test_multi_nonfinite_observation_stops_only_that_one():
    mp = synth.multi_gaussian(256, 1024, 8, 6, seed=3, snr_db=30.0)
    mp.Y[2, 17] = np.inf
    phi = torch.from_numpy(mp.phi).cuda()
    q1, q2 = q.quantize_pair(phi, 8, 1, q.STREAM_Q1, q.STREAM_Q2)
    ys = [q.quantize(torch.from_numpy(mp.Y[k]).cuda(), 8, 1, q.STREAM_Y) for k in range(6)]
    res = q.niht_solve_multi(q1, q2, ys, mp.s, 20)
    torch.cuda.synchronize()
    reps = res.all_reports()
    assert reps[2].status == q.ERR_NONFINITE and reps[2].iters_run == 0
    assert torch.all(res.x[2] == 0)
    assert all(reps[k].status == q.OK and reps[k].iters_run == 20 for k in (0, 1, 3, 4, 5))


def test_multi_zero_iterations_gives_initial_supports():
    mp = synth.multi_gaussian(256, 1024, 10, 5, seed=8)
    res, (q1, q2, ys) = _multi_run(mp, 8, 8, 0, seed=3)
    for k in range(5):
        sv = q.niht_solve(q1, q2, ys[k], mp.s, 0)
        torch.cuda.synchronize()
        assert torch.equal(torch.sort(sv.support).values, res.support[k])
        assert torch.all(res.x[k] == 0)


def test_multi_exact_ties_resolve_by_index():
    # +-1 columns duplicated: identical codes and gradients, ties at the s-th key broken by index;
    # every right-hand side the same observation, each against the oracle at every iteration
    p = synth.duplicated_pm1(256, 96, 4, 6, seed=3)
    Y = np.stack([p.y] * 3)
    mp = synth.MultiProblem(phi=p.phi, Y=Y, X_true=np.stack([p.x_true] * 3), s=p.s, name="dup")
    res, _ = _multi_run(mp, 8, 8, 12, seed=1)
    ref, _ = oracle.qiht(p.phi, p.y, p.s, 12, bits_phi=8, bits_y=8, seed=1, trace=True)
    for k in range(3):
        assert res.report(k).status == ref.status
        assert np.array_equal(res.support[k].cpu().numpy(), ref.support)
        x = res.x[k].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(x - ref.x) <= 1e-4 * np.linalg.norm(ref.x)
