"""The separable (MRI) operator with quantized transform factors (qiht_sep_quantize_factor,
qiht_sep_apply, qiht_niht_solve_separable) against the CPU oracle.

The oracle side materializes Phi-hat = S (A-hat (x) A-hat), stacked real, in FP64 from the oracle's
own quantization of the stacked factor [Re A; Im A] (a Kronecker product of its dequantized
codes), and runs Algorithm 2 on it with oracle.niht. The GPU applies the operator as FP32
transforms of the N x N image (two GEMMs per product and a gather or a scatter), so its
products carry FP32 accumulation error: for K-term sums in two stages,
  |err| <= (4N + 16) 2^-24 * mag,  mag = (|Ar| + |Ai|) |X| (|Ar| + |Ai|)^T  (forward; the
  adjoint's mag is the same form with |Zr| + |Zi|), which bounds every intermediate magnitude.
Solves follow the parity rule with the ambiguity gap at 1e-4 (FP32 products, not exact sums).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1802_04907_gb300 as q
import parity
import synth

pytestmark = pytest.mark.gpu

U = 2.0**-24


def _op(p):
    return q.SepOp(torch.from_numpy(p.meta["factor"]).cuda(), torch.from_numpy(p.meta["mask"]).cuda())


def _factor_hat(p, bits, seed, stream):
    codes, c = oracle.quantize(p.meta["factor"], bits, seed, stream)
    return codes, oracle.dequantize(codes, bits, c)


def _materialize(Fh, mask, N):
    A = Fh[:N] + 1j * Fh[N:]
    k1, k2 = mask // N, mask % N
    rows = (A[k1][:, :, None] * A[k2][:, None, :]).reshape(mask.size, N * N)
    return np.concatenate([rows.real, rows.imag])


@pytest.mark.parametrize("bits", [8, 12])
@pytest.mark.parametrize("N", [16, 32])
def test_sep_factor_codes(bits, N):
    p = synth.mri(N, s=8, seed=1)
    codes, fh, scale = q.sep_quantize_factor(_op(p), bits, 0xABC + bits, 1)
    want, c = oracle.quantize(p.meta["factor"], bits, 0xABC + bits, 1)
    assert scale.item() == c
    got = codes.cpu().numpy().view(np.uint16)
    assert np.array_equal(got, want)
    deq = oracle.dequantize(want, bits, c)
    assert np.all(np.abs(fh.cpu().numpy() - deq) <= 2.0**-23 * np.abs(deq))


def _mag_fwd(Fh, X, N):
    Aa = np.abs(Fh[:N]) + np.abs(Fh[N:])
    return Aa @ np.abs(X) @ Aa.T


@pytest.mark.parametrize("N", [16, 32, 64])
def test_sep_products(N):
    p = synth.mri(N, s=max(8, N * N // 32), seed=2)
    op = _op(p)
    bits = 12
    codes, Fh = _factor_hat(p, bits, 5, 0)
    _, fh_gpu, _ = q.sep_quantize_factor(op, bits, 5, 0)
    Phi = _materialize(Fh, p.meta["mask"], N)
    rng = np.random.Generator(np.random.PCG64(N))
    x = rng.standard_normal(N * N).astype(np.float32)
    x[rng.choice(N * N, N * N // 2, replace=False)] = 0.0
    r = rng.standard_normal(Phi.shape[0]).astype(np.float32)
    fwd = q.sep_apply(op, fh_gpu, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    adj = q.sep_apply(op, fh_gpu, torch.from_numpy(r).cuda(), adjoint=True).cpu().numpy().astype(np.float64)
    ref_f = Phi @ x.astype(np.float64)
    ref_a = Phi.T @ r.astype(np.float64)
    k1, k2 = p.meta["mask"] // N, p.meta["mask"] % N
    mf = _mag_fwd(Fh, x.reshape(N, N), N)[k1, k2]
    bound_f = (4 * N + 16) * U * np.concatenate([mf, mf]) + 1e-30
    assert np.all(np.abs(fwd - ref_f) <= bound_f), (np.abs(fwd - ref_f) / bound_f).max()
    M = p.meta["mask"].size
    Z = np.zeros((N, N))
    Z[k1, k2] = np.abs(r[:M]) + np.abs(r[M:])
    Aa = np.abs(Fh[:N]) + np.abs(Fh[N:])
    ma = (Aa.T @ Z @ Aa).reshape(-1)
    bound_a = (4 * N + 16) * U * ma + 1e-30
    assert np.all(np.abs(adj - ref_a) <= bound_a), (np.abs(adj - ref_a) / bound_a).max()


def test_sep_adjoint_identity_full_size():
    # the 128 x 128 operator (a third of k-space, 11364 stacked rows): <Phi-hat x, r> = <x, Phi-hat^T r>
    p = synth.mri(128, s=512, seed=0)
    op = _op(p)
    _, fh, _ = q.sep_quantize_factor(op, 12, 3, 0)
    rng = np.random.Generator(np.random.PCG64(3))
    x = torch.from_numpy(rng.standard_normal(op.cols).astype(np.float32)).cuda()
    r = torch.from_numpy(rng.standard_normal(op.rows).astype(np.float32)).cuda()
    fx = q.sep_apply(op, fh, x).double()
    ar = q.sep_apply(op, fh, r, adjoint=True).double()
    lhs, rhs = float(torch.dot(fx, r.double())), float(torch.dot(x.double(), ar))
    scale = float(torch.linalg.norm(fx) * torch.linalg.norm(r))
    assert abs(lhs - rhs) <= 1e-5 * scale, (lhs, rhs, scale)
    # sampled rows of the forward product against the oracle's materialized rows
    codes, Fh = _factor_hat(p, 12, 3, 0)
    N = 128
    A = Fh[:N] + 1j * Fh[N:]
    xn = x.cpu().numpy().astype(np.float64).reshape(N, N)
    mask = p.meta["mask"]
    M = mask.size
    out = fx.cpu().numpy()
    Aa = np.abs(Fh[:N]) + np.abs(Fh[N:])
    for b in rng.choice(M, 40, replace=False):
        k1, k2 = mask[b] // N, mask[b] % N
        v = A[k1] @ xn @ A[k2]
        mag = Aa[k1] @ np.abs(xn) @ Aa[k2]
        assert abs(out[b] - v.real) <= (4 * N + 16) * U * mag
        assert abs(out[M + b] - v.imag) <= (4 * N + 16) * U * mag


def _solve_pair(N, s, iters, bits_f, bits_y, seed, snr_db=30.0):
    p = synth.mri(N, s=s, seed=seed, snr_db=snr_db)
    sv = q.niht_solve_separable(_op(p), torch.from_numpy(p.y).cuda(), bits_f, bits_y, 9, s, iters, trace=True)
    torch.cuda.synchronize()
    _, F1 = _factor_hat(p, bits_f, 9, 0)
    _, F2 = _factor_hat(p, bits_f, 9, 1)
    cy, sy = oracle.quantize(p.y, bits_y, 9, 2)
    yq = oracle.dequantize(cy, bits_y, sy)
    Phi1, Phi2 = _materialize(F1, p.meta["mask"], N), _materialize(F2, p.meta["mask"], N)
    ref = oracle.niht(Phi1, Phi2, yq, s, iters, trace=True)
    return p, sv, ref


def _check(p, sv, ref, label):
    rep = sv.read_report()
    tr = {k: v.cpu().numpy() for k, v in sv.trace.items()}
    return parity.check(label, ref, p.x_true, x=sv.x.cpu().numpy(), support=sv.support.cpu().numpy(),
                        status=rep.status, iters_run=rep.iters_run, resid_norm2=rep.resid_norm2,
                        sup_trace=tr["support"], mu_trace=tr["mu"], resid_trace=tr["resid2"], gap=1e-4)


@pytest.mark.parametrize("N,s,bits_f,bits_y", [(32, 24, 12, 8), (32, 24, 8, 12), (64, 96, 12, 8)])
def test_sep_solve_against_oracle(N, s, bits_f, bits_y):
    p, sv, ref = _solve_pair(N, s, 40, bits_f, bits_y, seed=N + bits_f)
    _check(p, sv, ref, f"sep-{N}-{bits_f}/{bits_y}")


def test_sep_solve_full_size():
    # the 128 x 128 MRI-shaped instance (11364 x 16384), s = 512, 12-bit factor, 8-bit k-space,
    # 20 iterations, against the oracle on the materialized quantized operator
    p, sv, ref = _solve_pair(128, 512, 20, 12, 8, seed=0)
    _check(p, sv, ref, "sep-128-12/8")


def test_sep_solve_512_first_iteration():
    # the paper's MRI size, 512 x 512 (176028 stacked rows, 262144 coefficients, s = 4096), where the
    # threshold is the multi-CTA select and no m x n matrix can be formed: the first iteration
    # against FP64 products of the oracle's quantized factors (the initial support H_s(Phi-hat_1^T
    # y-hat), the step size on it and the residual after it)
    p = synth.mri(512, s=4096, seed=0, materialize=False)
    N, s = 512, 4096
    sv = q.niht_solve_separable(_op(p), torch.from_numpy(p.y).cuda(), 12, 8, 9, s, 1, trace=True)
    torch.cuda.synchronize()
    tr = {k: v.cpu().numpy() for k, v in sv.trace.items()}
    _, F1 = _factor_hat(p, 12, 9, 0)
    _, F2 = _factor_hat(p, 12, 9, 1)
    cy, sy = oracle.quantize(p.y, 8, 9, 2)
    yq = oracle.dequantize(cy, 8, sy)
    mask = p.meta["mask"]
    M = mask.size
    k1, k2 = mask // N, mask % N
    A1 = F1[:N] + 1j * F1[N:]
    A2 = F2[:N] + 1j * F2[N:]
    Z = np.zeros((N, N), complex)
    Z[k1, k2] = yq[:M] + 1j * yq[M:]
    g0 = (A1.T @ np.conj(Z) @ A1).real.reshape(-1)           # Phi-hat_1^T y-hat
    sup0, kth = oracle.top_s(g0, s)
    assert (kth[0] - kth[1]) / kth[0] > 1e-4                 # an unambiguous initial selection
    assert np.array_equal(tr["support"][0], sup0)
    # mu = ||g_G||^2 / ||Phi-hat_2 g_G||^2, then x1 = mu g on G and ||y-hat - Phi-hat_2 x1||^2
    X = np.zeros(N * N)
    X[sup0] = g0[sup0]
    B = A2 @ X.reshape(N, N) @ A2.T
    z = np.concatenate([B[k1, k2].real, B[k1, k2].imag])
    mu = float(g0[sup0] @ g0[sup0]) / float(z @ z)
    assert abs(tr["mu"][1] - mu) <= 1e-4 * mu, (tr["mu"][1], mu)
    assert np.array_equal(tr["support"][1], sup0)
    r1 = yq - mu * z
    assert abs(tr["resid2"][1] - float(r1 @ r1)) <= 1e-4 * float(r1 @ r1)
    rep = sv.read_report()
    assert rep.status == q.OK and rep.iters_run == 1
