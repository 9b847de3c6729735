"""CPU oracle of K unrolled QIHT iterations and their adjoint (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may import this
module. Plain numpy in FP64, written from the iteration of Algorithm 2; it shares no code
with the CUDA library.

The unrolled map (one problem). Phi1, Phi2 are the two quantized matrices (m x n, the
dequantized codes); a per-row complex gain g = a + i b scales the rows of the measurement
operator, stacked as a real system A_i = [diag(a); diag(b)] Phi_i (2m x n), as the complex
measurement of the radio-interferometry experiment is stacked (Section IV-B). With x_0 = 0:

    r_t = y - A2 x_t                     (2m)
    h_t = A1^T r_t                        (n)      the gradient of Algorithm 2
    G_t = supp H_s(h_0) for t = 0, supp x_t otherwise
    mu_t = ||P h_t||^2 / ||A2 P h_t||^2   (P: restriction to G_t; Eq. step_size)
    x_{t+1} = P_{t+1} (x_t + mu_t h_t),   G_{t+1} = supp H_s(x_t + mu_t h_t)

The support masks G_t are held fixed when differentiating (they are piecewise constant);
the unrolled layers use the adaptive step without the backtracking test. The adjoint
returns dL/dy, dL/da, dL/db for dL/dx_K given.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import top_s


def stacked(Phi: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """[diag(a); diag(b)] Phi (2m x n)."""
    return np.vstack([a[:, None] * Phi, b[:, None] * Phi])


@dataclass
class Step:
    x: np.ndarray        # x_t (n)
    r: np.ndarray        # r_t (2m)
    q: np.ndarray        # Phi2 x_t (m)
    h: np.ndarray        # h_t (n)
    G: np.ndarray        # G_t (s indices, ascending)
    u: np.ndarray        # Phi2 P h_t (m)
    N: float
    D: float
    mu: float
    Gn: np.ndarray       # G_{t+1}


def _top(v: np.ndarray, s: int) -> np.ndarray:
    sel, _ = top_s(v, s)
    return np.sort(sel)


def forward(Phi1, Phi2, y, a, b, s: int, K: int):
    """x_K and the record of every step."""
    Phi1 = np.asarray(Phi1, np.float64)
    Phi2 = np.asarray(Phi2, np.float64)
    y = np.asarray(y, np.float64)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    A1, A2 = stacked(Phi1, a, b), stacked(Phi2, a, b)
    n = Phi1.shape[1]
    x = np.zeros(n)
    steps = []
    G = None
    for t in range(K):
        q = Phi2 @ x
        r = y - A2 @ x
        h = A1.T @ r
        if t == 0:
            G = _top(h, s)                             # initial support of Algorithm 2
        Ph = np.zeros(n)
        Ph[G] = h[G]
        u = Phi2 @ Ph
        w = np.concatenate([a * u, b * u])
        N = float(Ph @ Ph)
        D = float(w @ w)
        mu = N / D if D > 0.0 else 0.0
        z = x + mu * h
        Gn = _top(z, s)
        xn = np.zeros(n)
        xn[Gn] = z[Gn]
        steps.append(Step(x=x, r=r, q=q, h=h, G=G, u=u, N=N, D=D, mu=mu, Gn=Gn))
        x = xn
        G = Gn
    return x, steps


def backward(Phi1, Phi2, a, b, steps, xbar_K):
    """(dL/dy, dL/da, dL/db) from dL/dx_K through the recorded steps (masks fixed)."""
    Phi1 = np.asarray(Phi1, np.float64)
    Phi2 = np.asarray(Phi2, np.float64)
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    A1, A2 = stacked(Phi1, a, b), stacked(Phi2, a, b)
    m, n = Phi1.shape
    xbar = np.asarray(xbar_K, np.float64).copy()
    ybar = np.zeros(2 * m)
    abar = np.zeros(m)
    bbar = np.zeros(m)
    for st in reversed(steps):
        v = np.zeros(n)
        v[st.Gn] = xbar[st.Gn]                        # through x_{t+1} = P_{t+1}(x_t + mu h)
        mubar = float(v @ st.h)
        Ph = np.zeros(n)
        Ph[st.G] = st.h[st.G]
        w = np.concatenate([a * st.u, b * st.u])
        hbar = st.mu * v
        if st.D > 0.0:
            c = A2.T @ w                               # d mu / d h = (2/D)(P h - mu P A2^T A2 P h)
            Pc = np.zeros(n)
            Pc[st.G] = c[st.G]
            hbar = hbar + mubar * (2.0 / st.D) * (Ph - st.mu * Pc)
            # mu through D = ||A2 P h||^2: A2bar += -(2 mubar mu / D) w (P h)^T
            coef = -2.0 * mubar * st.mu / st.D
            abar += coef * w[:m] * st.u
            bbar += coef * w[m:] * st.u
        p = Phi1 @ hbar                                # h = A1^T r: rbar = A1 hbar, A1bar += r hbar^T
        rbar = np.concatenate([a * p, b * p])
        abar += st.r[:m] * p
        bbar += st.r[m:] * p
        ybar += rbar                                   # r = y - A2 x: ybar += rbar, A2bar -= rbar x^T
        abar -= rbar[:m] * st.q
        bbar -= rbar[m:] * st.q
        xbar = v - A2.T @ rbar
    return ybar, abar, bbar


def loss_and_grads(Phi1, Phi2, y, a, b, s, K, x_true):
    """L = ||x_K - x_true||^2 and its gradients in y, a, b."""
    xK, steps = forward(Phi1, Phi2, y, a, b, s, K)
    d = xK - np.asarray(x_true, np.float64)
    gy, ga, gb = backward(Phi1, Phi2, a, b, steps, 2.0 * d)
    return float(d @ d), gy, ga, gb, xK, steps
