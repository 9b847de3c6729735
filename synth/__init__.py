"""Seeded synthetic workloads for QIHT (compressive sensing with quantized data).

This module only draws inputs: measurement matrices, sparse signals, noise and
observations. It holds none of the method's arithmetic (no quantizer, no
products with quantized matrices, no thresholding), so the CPU oracle and the
CUDA path can both consume exactly the same arrays.

Every generator takes an integer seed and uses numpy's PCG64 bit generator.

Workloads follow the shapes and distributions of the paper's experiments
(Section IV): Gaussian measurement matrices with i.i.d. entries (Section IV-A),
noisy observations at a stated SNR, and a radio-interferometry measurement
matrix built from antenna positions and a pixel grid (Section IV-B, radio
astronomy). The LOFAR recordings are not available, so the interferometry
workload is synthetic: random antenna layout, point sources at random pixels. The MRI
workload (Section IV-B, magnetic resonance imaging) samples k-space of a Haar-sparse
synthetic head image on radial lines; the paper's brain image is not available either.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One sparse recovery instance y = Phi x + e (Section I-A, Eq. 1)."""

    phi: np.ndarray | None   # float32, m x n, C order (row-major); None for an operator-only instance
    y: np.ndarray            # float32, m
    x_true: np.ndarray       # float64, n (s nonzeros)
    support: np.ndarray      # int64, sorted indices of the nonzeros of x_true
    s: int
    name: str
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.phi.shape[0]) if self.phi is not None else int(self.meta["rows"])

    @property
    def n(self) -> int:
        return int(self.phi.shape[1]) if self.phi is not None else int(self.meta["cols"])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _noise_sigma(clean: np.ndarray, snr_db: float) -> float:
    # SNR defined as 10 log10(||Phi x||^2 / ||e||^2) (Section IV-B, radio astronomy paragraph)
    m = clean.shape[0]
    return float(np.sqrt(np.dot(clean, clean) / (m * 10.0 ** (snr_db / 10.0))))


def gaussian(m: int, n: int, s: int, seed: int, *, snr_db: float | None = None,
             values: str = "normal", name: str | None = None) -> Problem:
    """Gaussian measurement matrix with entries N(0, 1/m) (Section IV-A data).

    values:
      "normal"  nonzeros of x drawn N(0, 1)                      (Section IV-A)
      "pm_u"    nonzeros +-U(0.5, 1.5) with random signs          (large single solve)
      "ones"    nonzeros equal to 1 (equal-magnitude case)        (Section IV-A)
    snr_db: None for noiseless y = Phi x, else Gaussian noise at that SNR.
    """
    rng = _rng(seed)
    phi = rng.standard_normal((m, n), dtype=np.float32)
    phi *= np.float32(1.0 / np.sqrt(m))
    support = np.sort(rng.choice(n, size=s, replace=False)).astype(np.int64)
    x = np.zeros(n, dtype=np.float64)
    if values == "normal":
        x[support] = rng.standard_normal(s)
    elif values == "pm_u":
        sign = np.where(rng.random(s) < 0.5, -1.0, 1.0)
        x[support] = sign * rng.uniform(0.5, 1.5, size=s)
    elif values == "ones":
        x[support] = 1.0
    else:
        raise ValueError(f"unknown values kind {values!r}")
    clean = phi[:, support].astype(np.float64) @ x[support]
    if snr_db is not None:
        clean = clean + _noise_sigma(clean, snr_db) * rng.standard_normal(m)
    return Problem(phi=phi, y=clean.astype(np.float32), x_true=x, support=support, s=s,
                   name=name or f"gaussian_{m}x{n}_s{s}",
                   meta={"snr_db": snr_db, "values": values, "seed": seed})


def interferometry(n_ant: int = 48, grid: int = 128, n_src: int = 50, s: int = 64,
                   snr_db: float = 20.0, seed: int = 0, *, wavelength_m: float = 5.0,
                   array_diameter_m: float = 1000.0, name: str | None = None) -> Problem:
    """Radio-interferometry shaped instance, stacked to a real system.

    Antennas are uniform in a disk of the given diameter. Every ordered pair
    (a, b), a != b, is one baseline with uv coordinates (p_a - p_b) / lambda.
    The sky is a grid x grid image of direction cosines (l, m) centred on 0
    with spacing lambda / (3 * diameter). The complex measurement matrix is
    Phi_kp = exp(-2 pi i (u_k l_p + v_k m_p)) (Section IV-B, radio astronomy),
    and the real and imaginary parts are stacked: [Re Phi; Im Phi] x = [Re y; Im y]
    with a real, nonnegative sky x.
    """
    rng = _rng(seed)
    radius = 0.5 * array_diameter_m
    r = radius * np.sqrt(rng.random(n_ant))
    th = 2.0 * np.pi * rng.random(n_ant)
    pos = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    a, b = np.meshgrid(np.arange(n_ant), np.arange(n_ant), indexing="ij")
    keep = a != b
    uv = (pos[a[keep]] - pos[b[keep]]) / wavelength_m          # (K, 2) in wavelengths
    dl = wavelength_m / (3.0 * array_diameter_m)
    coords = (np.arange(grid) - grid // 2) * dl
    lgrid, mgrid = np.meshgrid(coords, coords, indexing="ij")
    lm = np.stack([lgrid.ravel(), mgrid.ravel()], axis=1)      # (N, 2)
    phase = -2.0 * np.pi * (uv @ lm.T)                         # (K, N), fp64
    k = uv.shape[0]
    n = lm.shape[0]
    phi = np.empty((2 * k, n), dtype=np.float32)
    phi[:k] = np.cos(phase)
    phi[k:] = np.sin(phase)
    del phase
    src = np.sort(rng.choice(n, size=n_src, replace=False)).astype(np.int64)
    x = np.zeros(n, dtype=np.float64)
    x[src] = rng.lognormal(0.0, 1.0, size=n_src)
    clean = phi[:, src].astype(np.float64) @ x[src]
    # complex Gaussian noise: independent real and imaginary parts of equal variance
    sigma = _noise_sigma(clean, snr_db)
    y = clean + sigma * rng.standard_normal(2 * k)
    return Problem(phi=phi, y=y.astype(np.float32), x_true=x, support=src, s=s,
                   name=name or f"interferometry_{2 * k}x{n}_s{s}",
                   meta={"snr_db": snr_db, "n_ant": n_ant, "grid": grid, "n_src": n_src,
                         "seed": seed, "wavelength_m": wavelength_m})


def interferometry_gridded(n_ant: int = 48, grid: int = 128, n_src: int = 50, s: int = 64,
                           snr_db: float = 20.0, seed: int = 0, *, wavelength_m: float = 5.0,
                           array_diameter_m: float = 1000.0, materialize: bool = True,
                           name: str | None = None) -> Problem:
    """The interferometry instance of `interferometry` with gridded visibilities: every
    baseline's (u, v) is moved to the nearest point of the uv grid dual to the g x g sky grid
    (spacing 1 / (g dl) wavelengths), the usual gridding step of synthesis imaging. The phase of
    entry (k, p), p = ix g + iy, is then 2 pi t / g with the integer
      t = (u_k (ix - g/2) + v_k (iy - g/2)) mod g,
    so Phi is generated from the integer baselines and a table of 2g values:
      Phi[k][p] = table[t] = cos(2 pi t / g),  Phi[K + k][p] = table[g + t] = -sin(2 pi t / g).
    meta holds "uv" (int32, K x 2), "table" (float32, 2g) and "grid". K = n_ant (n_ant - 1)
    ordered pairs, cut to a multiple of four. materialize=False leaves phi as None (only the
    operator) for sizes whose dense matrix is not wanted; y is then formed from the sources'
    columns alone."""
    rng = _rng(seed)
    radius = 0.5 * array_diameter_m
    r = radius * np.sqrt(rng.random(n_ant))
    th = 2.0 * np.pi * rng.random(n_ant)
    pos = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    a, b = np.meshgrid(np.arange(n_ant), np.arange(n_ant), indexing="ij")
    keep = a != b
    uv = (pos[a[keep]] - pos[b[keep]]) / wavelength_m             # (K, 2) in wavelengths
    uv = uv[: uv.shape[0] - uv.shape[0] % 4]
    dl = wavelength_m / (3.0 * array_diameter_m)
    uvi = np.rint(uv * (grid * dl)).astype(np.int32)               # grid units
    K = uvi.shape[0]
    n = grid * grid
    tt = np.arange(grid, dtype=np.float64)
    table = np.concatenate([np.cos(2.0 * np.pi * tt / grid), -np.sin(2.0 * np.pi * tt / grid)]).astype(np.float32)
    off = np.arange(grid, dtype=np.int64) - grid // 2

    def columns(idx):
        ix, iy = idx // grid, idx % grid
        t = (uvi[:, :1].astype(np.int64) * off[ix][None, :] + uvi[:, 1:].astype(np.int64) * off[iy][None, :]) % grid
        return np.concatenate([table[t], table[grid + t]], axis=0)   # (2K, len(idx)) float32

    src = np.sort(rng.choice(n, size=n_src, replace=False)).astype(np.int64)
    x = np.zeros(n, dtype=np.float64)
    x[src] = rng.lognormal(0.0, 1.0, size=n_src)
    phi = None
    if materialize:
        phi = np.empty((2 * K, n), dtype=np.float32)
        for c0 in range(0, n, 4096):
            idx = np.arange(c0, min(n, c0 + 4096))
            phi[:, c0:c0 + idx.size] = columns(idx)
    clean = columns(src).astype(np.float64) @ x[src]
    sigma = _noise_sigma(clean, snr_db)
    y = clean + sigma * rng.standard_normal(2 * K)
    return Problem(phi=phi, y=y.astype(np.float32), x_true=x, support=src, s=s,
                   name=name or f"interferometry_gridded_{2 * K}x{n}_s{s}",
                   meta={"snr_db": snr_db, "n_ant": n_ant, "grid": grid, "n_src": n_src, "seed": seed,
                         "uv": uvi, "table": table, "rows": 2 * K, "cols": n})


def haar_synthesis(N: int) -> np.ndarray:
    """Orthonormal multilevel 1D Haar basis as an N x N synthesis matrix (N a power of two): a
    signal is H^T-analysed to coefficients c = H v and rebuilt as v = H^T c. Built by the usual
    recursion: the rows of H_2N are the rows of H_N with every entry duplicated (coarse
    functions), then the N finest differences, all scaled by 1/sqrt(2)."""
    if N < 1 or N & (N - 1):
        raise ValueError("N must be a power of two")
    H = np.ones((1, 1))
    while H.shape[0] < N:
        k = H.shape[0]
        coarse = np.kron(H, np.array([[1.0, 1.0]]))
        fine = np.kron(np.eye(k), np.array([[1.0, -1.0]]))
        H = np.vstack([coarse, fine]) / np.sqrt(2.0)
    return H.T                                   # columns = basis vectors (synthesis)


def radial_mask(N: int, fraction: float = 1.0 / 3.0) -> np.ndarray:
    """k-space positions (k1, k2) in DFT index order (0 .. N-1) on radial lines through the
    centre, closed under reflection through the centre, with as few equally spaced lines as
    reach the given fraction of the N x N grid (the paper undersamples k-space by a factor of 3
    with a radial mask, Section IV-B)."""
    c = N // 2
    r = np.arange(-c, c, 0.5)
    for lines in range(1, 4 * N):
        th = np.pi * np.arange(lines) / lines
        u = np.rint(np.outer(np.cos(th), r)).astype(np.int64).ravel()
        v = np.rint(np.outer(np.sin(th), r)).astype(np.int64).ravel()
        keep = (u >= -c) & (u <= c) & (v >= -c) & (v <= c)
        u, v = u[keep] % N, v[keep] % N
        # with each position its reflection through the centre (the k-space of a real image is
        # conjugate-symmetric, and the lines pass through the centre)
        pos = np.unique(np.concatenate([u * N + v, ((-u) % N) * N + ((-v) % N)]))
        if pos.size >= fraction * N * N:
            return np.stack([pos // N, pos % N], axis=1)
    raise RuntimeError("mask fraction not reached")


def head_phantom(N: int) -> np.ndarray:
    """A piecewise-constant head-like image (N x N): an outer shell, a darker interior and a few
    small ellipses of different intensities (a stand-in for the paper's brain image)."""
    yy, xx = np.mgrid[-1:1:complex(0, N), -1:1:complex(0, N)]
    img = np.zeros((N, N))
    # (intensity, centre x, centre y, half axis a, half axis b, angle in degrees)
    for val, x0, y0, a, b, ang in [(1.0, 0.0, 0.0, 0.70, 0.92, 0), (-0.75, 0.0, -0.02, 0.65, 0.86, 0),
                                   (-0.2, 0.2, 0.05, 0.12, 0.30, -16), (-0.2, -0.22, 0.05, 0.16, 0.38, 16),
                                   (0.15, 0.0, 0.38, 0.22, 0.26, 0), (0.1, 0.0, -0.55, 0.05, 0.05, 0),
                                   (0.1, -0.08, -0.6, 0.05, 0.025, 0), (0.1, 0.06, -0.6, 0.025, 0.05, 0),
                                   (0.12, 0.3, -0.25, 0.06, 0.1, 30)]:
        t = np.deg2rad(ang)
        xr = (xx - x0) * np.cos(t) + (yy - y0) * np.sin(t)
        yr = -(xx - x0) * np.sin(t) + (yy - y0) * np.cos(t)
        img[(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] += val
    return img


def mri(grid: int = 128, s: int = 512, snr_db: float = 30.0, seed: int = 0, *,
        fraction: float = 1.0 / 3.0, materialize: bool = True, name: str | None = None) -> Problem:
    """MRI-shaped instance (Section IV-B, magnetic resonance imaging), stacked to a real system.

    Phi = S F W^-1: W^-1 the 2D orthonormal Haar synthesis (tensor product of the 1D basis of
    haar_synthesis), F the orthonormal 2D DFT, S the radial k-space mask of radial_mask (a third
    of the grid). With A = F_1 H^T (N x N, unitary), the k-space sample at (k1, k2) of the
    coefficient image C is sum A[k1, j1] A[k2, j2] C[j1, j2], so the row of Phi for that sample
    is kron(A[k1], A[k2]) over the coefficient index j1 N + j2. The real and imaginary parts are
    stacked: [Re Phi; Im Phi] x = [Re y; Im y]. x is the s largest Haar coefficients of
    head_phantom (exactly s-sparse); y = Phi x + complex Gaussian noise at the given SNR. The
    paper's brain image and SparseMRI are not available, so the image is synthetic. meta holds
    the operator form too: "factor" = [Re A; Im A] (float32, 2N x N) and "mask" = k1 N + k2 of
    every row (int32, in row order). materialize=False leaves phi as None (the paper's 512 x 512
    size would need ~180 GB) and forms y through the transforms.
    """
    N = grid
    H = haar_synthesis(N)
    F = np.exp(-2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N) / np.sqrt(N)
    A = F @ H                                            # N x N, unitary
    ks = radial_mask(N, fraction)
    k = ks.shape[0]
    n = N * N
    phi = None
    if materialize:
        phi = np.empty((2 * k, n), dtype=np.float32)
        for b0 in range(0, k, 512):
            b1 = min(k, b0 + 512)
            rows = (A[ks[b0:b1, 0]][:, :, None] * A[ks[b0:b1, 1]][:, None, :]).reshape(b1 - b0, n)
            phi[b0:b1] = rows.real
            phi[k + b0:k + b1] = rows.imag
    coef = H.T @ head_phantom(N) @ H                     # analysis: C = H_a X H_a^T, H_a = H^T
    flat = coef.ravel()
    support = np.sort(np.argsort(-np.abs(flat), kind="stable")[:s]).astype(np.int64)
    x = np.zeros(n)
    x[support] = flat[support]
    if materialize:
        clean = phi[:, support].astype(np.float64) @ x[support]
    else:
        # the same samples through the transforms: B = A X A^T read at the mask
        B = A @ x.reshape(N, N) @ A.T
        b = B[ks[:, 0], ks[:, 1]]
        clean = np.concatenate([b.real, b.imag])
    rng = _rng(seed)
    y = clean + _noise_sigma(clean, snr_db) * rng.standard_normal(2 * k)
    return Problem(phi=phi, y=y.astype(np.float32), x_true=x, support=support, s=s,
                   name=name or f"mri_{2 * k}x{n}_s{s}",
                   meta={"snr_db": snr_db, "grid": N, "fraction": fraction, "samples": k, "seed": seed,
                         "rows": 2 * k, "cols": n,
                         "factor": np.concatenate([A.real, A.imag]).astype(np.float32),
                         "mask": (ks[:, 0] * N + ks[:, 1]).astype(np.int32)})


# Named workloads (sizes from the configurations this library is measured on).
def duplicated_pm1(m: int, base: int, dup: int, s: int, seed: int) -> Problem:
    """Phi with +-1 entries whose `base` distinct columns each appear `dup` times in a row
    (column k * dup + d is distinct column k); x has s nonzeros +-U(0.5, 1.5), each on copy 2
    (or the last copy) of a distinct column; y = Phi x (noiseless). Entries +-1 sit on the
    quantizer's end levels, so duplicated columns keep identical codes: a workload with exact
    ties in the gradient."""
    rng = _rng(seed)
    cols = rng.choice(np.array([-1.0, 1.0], dtype=np.float32), size=(m, base))
    phi = np.ascontiguousarray(np.repeat(cols, dup, axis=1))
    picks = np.sort(rng.choice(base, size=s, replace=False))
    support = picks * dup + min(2, dup - 1)
    x = np.zeros(base * dup)
    x[support] = rng.uniform(0.5, 1.5, size=s) * rng.choice([-1.0, 1.0], size=s)
    y = (phi.astype(np.float64) @ x).astype(np.float32)
    return Problem(phi=phi, y=y, x_true=x, support=support.astype(np.int64), s=s,
                   name=f"duplicated_pm1_{m}x{base * dup}_s{s}_seed{seed}")


def batch_gaussian(count: int, seed: int, *, m_range=(128, 2048), n_per_m: int = 4, s_range=(8, 128),
                   snr_db: float | None = None, values: str = "normal") -> list:
    """Independent Gaussian problems of uneven sizes (the batched workload): m uniform in
    m_range, n = n_per_m m, s uniform in s_range (at most m), each drawn by gaussian()
    with its own seed."""
    rng = _rng(seed)
    out = []
    for i in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        s = int(min(m, rng.integers(s_range[0], s_range[1] + 1)))
        out.append(gaussian(m, n_per_m * m, s, seed=int(rng.integers(0, 2**31 - 1)), snr_db=snr_db, values=values,
                            name=f"batch{seed}_{i}"))
    return out


@dataclass
class MultiProblem:
    """Many observations of one matrix: Y[k] = Phi X[k] + E[k] (rows of Y and X)."""

    phi: np.ndarray          # float32, m x n
    Y: np.ndarray            # float32, nrhs x m
    X_true: np.ndarray       # float64, nrhs x n (s nonzeros per row)
    s: int
    name: str

    def problem(self, k: int) -> Problem:
        sup = np.flatnonzero(self.X_true[k])
        return Problem(phi=self.phi, y=self.Y[k], x_true=self.X_true[k], support=sup, s=self.s,
                       name=f"{self.name}_rhs{k}")


def multi_gaussian(m: int, n: int, s: int, nrhs: int, seed: int, *, snr_db: float | None = None,
                   values: str = "normal") -> MultiProblem:
    """One Gaussian Phi (entries N(0, 1/m)) and nrhs independent s-sparse signals with their
    observations (the many-right-hand-sides workload): supports uniform without replacement,
    nonzeros as in gaussian(), noise per observation at snr_db."""
    rng = _rng(seed)
    phi = rng.standard_normal((m, n), dtype=np.float32)
    phi *= np.float32(1.0 / np.sqrt(m))
    X = np.zeros((nrhs, n))
    Y = np.zeros((nrhs, m), dtype=np.float32)
    for k in range(nrhs):
        sup = np.sort(rng.choice(n, size=s, replace=False))
        if values == "normal":
            X[k, sup] = rng.standard_normal(s)
        elif values == "pm_u":
            X[k, sup] = np.where(rng.random(s) < 0.5, -1.0, 1.0) * rng.uniform(0.5, 1.5, size=s)
        elif values == "ones":
            X[k, sup] = 1.0
        else:
            raise ValueError(f"unknown values kind {values!r}")
        clean = phi[:, sup].astype(np.float64) @ X[k, sup]
        if snr_db is not None:
            clean = clean + _noise_sigma(clean, snr_db) * rng.standard_normal(m)
        Y[k] = clean.astype(np.float32)
    return MultiProblem(phi=phi, Y=Y, X_true=X, s=s, name=f"multi_{m}x{n}_s{s}_r{nrhs}")


def small_noiseless(seed: int = 0) -> Problem:
    """m=256, n=1024, s=16, N(0,1) nonzeros, noiseless (shape of Section IV-A)."""
    return gaussian(256, 1024, 16, seed, snr_db=None, values="normal", name="gaussian_256x1024_s16")


def large_noisy(seed: int = 0, m: int = 8192, n: int = 32768, s: int = 256) -> Problem:
    """m=8192, n=32768, s=256, +-U(0.5,1.5) nonzeros, 30 dB SNR."""
    return gaussian(m, n, s, seed, snr_db=30.0, values="pm_u", name=f"gaussian_{m}x{n}_s{s}_30dB")


def tiny(m: int, n: int, s: int, seed: int, snr_db: float | None = None) -> Problem:
    """Small Gaussian instance for brute-force checks (n <= 16)."""
    return gaussian(m, n, s, seed, snr_db=snr_db, values="normal", name=f"tiny_{m}x{n}_s{s}")


def random_floats(shape, seed: int, scale: float = 1.0, dtype=np.float32) -> np.ndarray:
    """Plain N(0, scale^2) array (for kernel-level tests)."""
    rng = _rng(seed)
    return (scale * rng.standard_normal(shape)).astype(dtype)
