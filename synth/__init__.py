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
workload is synthetic: random antenna layout, point sources at random pixels.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One sparse recovery instance y = Phi x + e (Section I-A, Eq. 1)."""

    phi: np.ndarray          # float32, m x n, C order (row-major)
    y: np.ndarray            # float32, m
    x_true: np.ndarray       # float64, n (s nonzeros)
    support: np.ndarray      # int64, sorted indices of the nonzeros of x_true
    s: int
    name: str
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.phi.shape[0])

    @property
    def n(self) -> int:
        return int(self.phi.shape[1])


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
