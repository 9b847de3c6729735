"""The interferometry workload generator (synth.interferometry) pinned to its definition:
unit-modulus complex entries, the antisymmetry of the baselines (the measurement of baseline
(a, b) is the conjugate of that of (b, a)), the origin pixel's column, a row against the
visibility phase computed from the antenna positions, and the noise level."""
import numpy as np

import synth


def test_entries_have_unit_modulus_and_conjugate_baseline_pairs():
    p = synth.interferometry(n_ant=6, grid=16, n_src=3, s=4, snr_db=20.0, seed=1)
    k = p.m // 2
    re, im = p.phi[:k].astype(np.float64), p.phi[k:].astype(np.float64)
    assert np.allclose(re ** 2 + im ** 2, 1.0, atol=1e-6)
    # ordered pairs (a, b), a != b, in row-major order of the antenna grid
    pairs = [(a, b) for a in range(6) for b in range(6) if a != b]
    assert k == len(pairs) == 30
    row = {pr: i for i, pr in enumerate(pairs)}
    for a, b in [(0, 1), (2, 5), (4, 3)]:
        i, j = row[(a, b)], row[(b, a)]
        assert np.allclose(re[i], re[j], atol=1e-6) and np.allclose(im[i], -im[j], atol=1e-6)


def test_origin_pixel_and_one_row_from_the_geometry():
    n_ant, grid, wl, diam = 5, 8, 5.0, 1000.0
    p = synth.interferometry(n_ant=n_ant, grid=grid, n_src=2, s=2, snr_db=20.0, seed=3,
                             wavelength_m=wl, array_diameter_m=diam)
    k = p.m // 2
    origin = (grid // 2) * grid + grid // 2           # l = m = 0
    assert np.allclose(p.phi[:k, origin], 1.0) and np.allclose(p.phi[k:, origin], 0.0)
    # the antenna layout is the generator's first draws: rebuild it and one visibility row
    rng = np.random.Generator(np.random.PCG64(3))
    r = 0.5 * diam * np.sqrt(rng.random(n_ant))
    th = 2.0 * np.pi * rng.random(n_ant)
    pos = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    u, v = (pos[0] - pos[1]) / wl                     # baseline (0, 1) is row 0
    dl = wl / (3.0 * diam)
    coords = (np.arange(grid) - grid // 2) * dl
    l, mm = np.meshgrid(coords, coords, indexing="ij")
    vis = np.exp(-2j * np.pi * (u * l.ravel() + v * mm.ravel()))
    assert np.allclose(p.phi[0], vis.real, atol=1e-6) and np.allclose(p.phi[k], vis.imag, atol=1e-6)


def test_sources_and_noise():
    p = synth.interferometry(n_ant=12, grid=32, n_src=6, s=8, snr_db=20.0, seed=2)
    assert np.count_nonzero(p.x_true) == 6 and np.all(p.x_true >= 0)
    clean = p.phi.astype(np.float64) @ p.x_true
    e = p.y.astype(np.float64) - clean
    assert abs(10.0 * np.log10(clean @ clean / (e @ e)) - 20.0) < 1.0
