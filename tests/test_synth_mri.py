"""The MRI-shaped workload generator (synth.mri) pinned to library transforms and definitions:
the Haar basis against its N = 2 definition and orthonormality; every row of Phi against
numpy's FFT of the image synthesized from the coefficients; the radial mask's symmetry and
fraction; the sparse x and the noise level."""
import numpy as np

import synth


def test_haar_basis():
    H2 = synth.haar_synthesis(2)
    assert np.allclose(H2, np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0))
    for N in (8, 64):
        H = synth.haar_synthesis(N)
        assert np.allclose(H.T @ H, np.eye(N), atol=1e-12)
        assert np.allclose(H[:, 0], 1.0 / np.sqrt(N))           # the scaling function
        # a piecewise-constant signal on dyadic halves has two nonzero coefficients
        v = np.r_[np.ones(N // 2), -2.0 * np.ones(N // 2)]
        assert np.count_nonzero(np.abs(H.T @ v) > 1e-12) == 2


def test_rows_are_sampled_fft_of_the_synthesized_image():
    N, s = 16, 20
    p = synth.mri(grid=N, s=s, snr_db=30.0, seed=3)
    ks = synth.radial_mask(N)
    k = ks.shape[0]
    assert p.phi.shape == (2 * k, N * N)
    H = synth.haar_synthesis(N)
    rng = np.random.Generator(np.random.PCG64(9))
    for _ in range(3):
        c = rng.standard_normal(N * N)
        img = H @ c.reshape(N, N) @ H.T                        # synthesis of the coefficient image
        K = np.fft.fft2(img) / N                              # orthonormal 2D DFT
        want = K[ks[:, 0], ks[:, 1]]
        got = p.phi.astype(np.float64) @ c
        assert np.allclose(got[:k], want.real, atol=1e-5) and np.allclose(got[k:], want.imag, atol=1e-5)


def test_radial_mask():
    for N in (16, 32, 128):
        ks = synth.radial_mask(N)
        pos = set(map(tuple, ks))
        assert (0, 0) in pos
        assert all(((-a) % N, (-b) % N) in pos for a, b in pos)   # symmetric through the centre
        frac = len(pos) / (N * N)
        assert 1.0 / 3.0 <= frac < 0.5, frac
        assert len(pos) == ks.shape[0]


def test_sparse_coefficients_and_noise():
    N, s = 32, 40
    p = synth.mri(grid=N, s=s, snr_db=20.0, seed=5)
    H = synth.haar_synthesis(N)
    coef = (H.T @ synth.head_phantom(N) @ H).ravel()
    assert np.count_nonzero(p.x_true) == s and len(p.support) == s
    assert np.allclose(p.x_true[p.support], coef[p.support])
    assert np.abs(coef[p.support]).min() >= np.sort(np.abs(coef))[-s] - 1e-12
    clean = p.phi.astype(np.float64) @ p.x_true
    e = p.y.astype(np.float64) - clean
    snr = 10.0 * np.log10(clean @ clean / (e @ e))
    assert abs(snr - 20.0) < 1.5, snr
