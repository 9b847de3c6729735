"""CPU oracle for QIHT (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
import this package. It wraps the plain C implementation in qiht_oracle.c
(FP64; the dense products and the quantizer split their outputs over OpenMP
threads without changing any sum) with ctypes and numpy. It shares no code with the CUDA
library of the package and never imports it.

Functions mirror the paper's steps:
  philox4x32_10, uniform         random numbers of the stochastic quantizer
  absmax                         c_v = max |v| (Appendix, quantization lemma)
  levels                         grid size: 2^b (Section III-A) or 2^(b-1)+1 (Appendix remark)
  quantize / dequantize          Q(v, b) of Section III-A, and its value c * q_code
  gemv_t, gemv_cols              plain FP64 products
  top_s                          hard threshold H_s (Eq. NIHT)
  step_size                      the step size's numerator and denominator (Eq. step_size;
                                 Algorithm 2's cross product of two realizations, or the
                                 forward square)
  niht, niht_seq                 Algorithm 2 (Algorithm 1 when both matrices are Phi); niht_seq
                                 with one realization per iteration (qiht_fresh)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qiht_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libqiht_oracle.so")

# status codes of the oracle (same numbering as the CUDA library's, compared in tests)
OK, ERR_ARG, ERR_BITS, ERR_NONFINITE, ERR_BACKTRACK_CAP = 0, 1, 2, 3, 5


def build(force: bool = False, mutant: int = 0, out: str | None = None) -> str:
    """Compile qiht_oracle.c into a shared library (gcc, no FMA contraction).

    mutant != 0 builds a variant with one deliberate mistake (mutation tests only)."""
    lib_path = out or (_LIB if mutant == 0 else os.path.join(_HERE, "_build", f"libqiht_oracle_m{mutant}.so"))
    os.makedirs(os.path.dirname(lib_path), exist_ok=True)
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= os.path.getmtime(_SRC):
        return lib_path
    tmp = lib_path + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           f"-DQO_MUTANT={int(mutant)}", "-o", tmp, _SRC, "-lm"]
    # OpenMP splits outputs over threads (results do not depend on the thread count); a
    # compiler without it builds the same code single-threaded
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, lib_path)
    return lib_path


_lib = None


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("c", ctypes.c_double), ("max_backtrack", ctypes.c_int32),
                ("mu_mode", ctypes.c_int32), ("tol", ctypes.c_double), ("grad_e4m3", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class _Trace(ctypes.Structure):
    _fields_ = [("support", ctypes.c_void_p), ("kth", ctypes.c_void_p), ("min_gap", ctypes.c_void_p),
                ("mu", ctypes.c_void_p), ("bt", ctypes.c_void_p), ("min_margin", ctypes.c_void_p),
                ("resid2", ctypes.c_void_p), ("x", ctypes.c_void_p), ("mu_fallback", ctypes.c_void_p),
                ("num", ctypes.c_void_p), ("xnorm2", ctypes.c_void_p)]


MU_FORWARD_SQ, MU_CROSS = 0, 1


def _mu_mode(mode) -> int:
    if mode in (0, "forward", "forward_sq"):
        return MU_FORWARD_SQ
    if mode in (1, "cross"):
        return MU_CROSS
    raise ValueError(f"mu_mode {mode!r}")


class _Report(ctypes.Structure):
    _fields_ = [("iters_run", ctypes.c_int32), ("backtracks", ctypes.c_int32),
                ("support_changes", ctypes.c_int32), ("status", ctypes.c_int32),
                ("resid_norm2", ctypes.c_double), ("mu", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        # QIHT_ORACLE_LIB points the wrapper at another build (mutation tests only)
        path = os.environ.get("QIHT_ORACLE_LIB") or build()
        # idle OpenMP threads sleep instead of spinning (the oracle runs beside GPU work)
        os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.qo_philox4x32_10.argtypes = [P, P, P]
        L.qo_philox4x32_10.restype = None
        L.qo_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
        L.qo_uniform.restype = ctypes.c_float
        L.qo_absmax.argtypes = [P, ctypes.c_int64, P]
        L.qo_absmax.restype = ctypes.c_float
        L.qo_quantize.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                  ctypes.c_uint32, ctypes.c_float, P]
        L.qo_quantize.restype = ctypes.c_int
        L.qo_dequantize.argtypes = [P, ctypes.c_int64, ctypes.c_int, ctypes.c_float, P]
        L.qo_dequantize.restype = None
        L.qo_gemv_t.argtypes = [P, P, ctypes.c_int64, ctypes.c_int64, P]
        L.qo_gemv_t.restype = None
        L.qo_gemv_cols.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, P, ctypes.c_int64, P]
        L.qo_gemv_cols.restype = None
        L.qo_top_s.argtypes = [P, ctypes.c_int32, ctypes.c_int32, P, P]
        L.qo_top_s.restype = None
        L.qo_niht.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                              ctypes.POINTER(_Params), P, P, ctypes.POINTER(_Trace),
                              ctypes.POINTER(_Report)]
        L.qo_niht.restype = ctypes.c_int
        L.qo_niht_seq.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.POINTER(_Params), P, P, ctypes.POINTER(_Trace), ctypes.POINTER(_Report)]
        L.qo_niht_seq.restype = ctypes.c_int
        L.qo_step_size.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, P, P, ctypes.c_int32, ctypes.c_int32, P, P,
                                   P, P]
        L.qo_step_size.restype = None
        L.qo_e4m3.argtypes = [ctypes.c_double]
        L.qo_e4m3.restype = ctypes.c_double
        L.qo_e4m3_terms.argtypes = [P, ctypes.c_int64, ctypes.c_int, P]
        L.qo_e4m3_terms.restype = None
        L.qo_set_threads.argtypes = [ctypes.c_int]
        L.qo_set_threads.restype = None
        L.qo_get_threads.argtypes = []
        L.qo_get_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def philox4x32_10(counter, key) -> np.ndarray:
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().qo_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(seed: int, stream: int, e: int) -> float:
    return float(lib().qo_uniform(seed, stream, e))


def absmax(v: np.ndarray) -> tuple[float, int]:
    v = np.ascontiguousarray(v, dtype=np.float32)
    bad = ctypes.c_int64(0)
    c = lib().qo_absmax(_ptr(v), v.size, ctypes.addressof(bad))
    return float(np.float32(c)), int(bad.value)


def levels(bits: int, odd: bool = False) -> int:
    """Number of quantization levels of b bits: 2^b equally spaced levels on [-1, 1]
    (Section III-A), or, with odd=True, the 2^(b-1) + 1 levels of spacing 1/2^(b-2)
    that the Appendix's remark on fixed-point hardware uses (0 is then a level)."""
    return 2 ** (bits - 1) + 1 if odd else 2**bits


def quantize(v: np.ndarray, bits: int, seed: int, stream: int, scale: float | None = None, *,
             row0: int = 0, col0: int = 0, rows_total: int | None = None,
             odd: bool = False) -> tuple[np.ndarray, float]:
    """Q(v, b) elementwise on a matrix (m x n) or vector (m,). Returns (codes, scale).

    codes have the shape of v (uint16). scale is c = max |v| unless given (for
    a block of a larger matrix, pass the whole matrix's scale, the block's
    position and the whole matrix's row count). odd selects the grid of
    levels(bits, odd=True).
    """
    v = np.asarray(v, dtype=np.float32)
    vec = v.ndim == 1
    v2 = np.ascontiguousarray(v.reshape(-1, 1) if vec else v)
    rows, cols = v2.shape
    if scale is None:
        scale, bad = absmax(v2)
        if bad:
            raise ValueError("non-finite input")
    codes = np.zeros((rows, cols), dtype=np.uint16)
    st = lib().qo_quantize(_ptr(v2), rows, cols, cols, row0, col0,
                           rows if rows_total is None else rows_total,
                           levels(bits, odd), seed, stream, np.float32(scale), _ptr(codes))
    if st != OK:
        raise ValueError(f"qo_quantize status {st}")
    return (codes.reshape(-1) if vec else codes), float(np.float32(scale))


def dequantize(codes: np.ndarray, bits: int, scale: float, *, odd: bool = False) -> np.ndarray:
    c = np.ascontiguousarray(codes, dtype=np.uint16)
    out = np.zeros(c.shape, dtype=np.float64)
    lib().qo_dequantize(_ptr(c), c.size, levels(bits, odd), np.float32(scale), _ptr(out))
    return out


def gemv_t(A: np.ndarray, r: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    m, n = A.shape
    g = np.zeros(n, dtype=np.float64)
    lib().qo_gemv_t(_ptr(A), _ptr(r), m, n, _ptr(g))
    return g


def gemv_cols(A: np.ndarray, idx: np.ndarray, v: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    m, n = A.shape
    z = np.zeros(m, dtype=np.float64)
    lib().qo_gemv_cols(_ptr(A), m, n, _ptr(idx), _ptr(v), idx.size, _ptr(z))
    return z


def set_threads(n: int) -> None:
    """Threads of the OpenMP split of the products and the quantizer (results are the same for
    any count)."""
    lib().qo_set_threads(int(n))


def get_threads() -> int:
    return int(lib().qo_get_threads())


def step_size(A1: np.ndarray, A2: np.ndarray, support: np.ndarray, g: np.ndarray, mu_mode=0) -> dict:
    """The step size's parts on support G (Eq. step_size, Algorithm 2): num = ||g_G||^2 and the
    denominator used: ||A2_G g_G||^2 (mu_mode "forward"), or the cross product
    (A1_G g_G)^T (A2_G g_G) of the two realizations (mu_mode "cross"), which falls back to the
    forward square when not positive."""
    A1 = np.ascontiguousarray(A1, dtype=np.float64)
    A2 = np.ascontiguousarray(A2, dtype=np.float64)
    sup = np.ascontiguousarray(support, dtype=np.int32)
    g = np.ascontiguousarray(g, dtype=np.float64)
    m, n = A2.shape
    out = np.zeros(4)
    coef = np.zeros(max(sup.size, 1))
    z1, z2 = np.zeros(m), np.zeros(m)
    lib().qo_step_size(_ptr(A1), _ptr(A2), m, n, _ptr(sup), _ptr(g), sup.size, _mu_mode(mu_mode), _ptr(out),
                       _ptr(coef), _ptr(z1), _ptr(z2))
    return {"num": out[0], "den": out[1], "cross": out[2], "fallback": bool(out[3])}


def e4m3(v) -> np.ndarray:
    """Nearest E4M3 values (OCP 8-bit floating point: bias 7, 3 fraction bits, subnormals,
    largest finite 448), ties to even, saturating at 448; elementwise."""
    v = np.asarray(v, dtype=np.float64)
    return np.vectorize(lambda t: lib().qo_e4m3(float(t)), otypes=[np.float64])(v) if v.size else v.copy()


def e4m3_terms(r: np.ndarray, terms: int = 3) -> np.ndarray:
    """r held as 2^e (t_1 + ... + t_terms): max |r| 2^-e in [2^7, 2^8), t_k the E4M3 value
    nearest to what t_1 .. t_{k-1} leave of r 2^-e."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros_like(r)
    lib().qo_e4m3_terms(_ptr(r), r.size, int(terms), _ptr(out))
    return out


def top_s(a: np.ndarray, s: int) -> tuple[np.ndarray, np.ndarray]:
    a = np.ascontiguousarray(a, dtype=np.float64)
    sel = np.zeros(s, dtype=np.int32)
    kth = np.zeros(2, dtype=np.float64)
    lib().qo_top_s(_ptr(a), a.size, s, _ptr(sel), _ptr(kth))
    return sel, kth


@dataclass
class NihtResult:
    x: np.ndarray
    support: np.ndarray
    status: int
    iters_run: int
    backtracks: int
    support_changes: int
    resid_norm2: float
    mu: float
    trace: dict | None


def niht(A1: np.ndarray, A2: np.ndarray, y: np.ndarray, s: int, iters: int, *, k: float = 2.0,
         c: float = 0.01, max_backtrack: int = 32, mu_mode=0, tol: float = 0.0, grad_e4m3: bool = False,
         trace: bool | str = False) -> NihtResult:
    """Algorithm 2 with matrices A1 (for g = A1^T r) and A2 (for A2 x, mu, omega), FP64.

    mu_mode "cross" takes Algorithm 2's printed step-size denominator (see step_size); tol > 0
    stops after the first iteration whose ||y - A2 x||^2 <= tol; grad_e4m3 forms every gradient
    from the residual (and y) held as three e4m3 terms (see e4m3_terms).
    trace=True records supports, gaps, step sizes and residuals per iteration;
    trace="x" also records every iterate."""
    return niht_seq([A1], [A2], [y], s, iters, k=k, c=c, max_backtrack=max_backtrack, mu_mode=mu_mode, tol=tol,
                    grad_e4m3=grad_e4m3, trace=trace)


def niht_seq(A1s: list, A2s: list, ys: list, s: int, iters: int, *, k: float = 2.0, c: float = 0.01,
             max_backtrack: int = 32, mu_mode=0, tol: float = 0.0, grad_e4m3: bool = False,
             trace: bool | str = False) -> NihtResult:
    """Algorithm 2 with one realization per iteration: iteration t (1..iters) uses A1s[t], A2s[t],
    ys[t]; index 0 gives the initial support. Lists of length 1 repeat their one entry."""
    def full(lst):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in lst]
        return arrs if len(arrs) > 1 else arrs * (iters + 1)
    A1l, A2l, yl = full(A1s), full(A2s), full(ys)
    assert len(A1l) == len(A2l) == len(yl) == iters + 1
    A1 = A1l[0]
    m, n = A1.shape
    x = np.zeros(n, dtype=np.float64)
    sup = np.zeros(s, dtype=np.int32)
    p = _Params(k, c, max_backtrack, _mu_mode(mu_mode), float(tol), int(bool(grad_e4m3)), 0)
    rep = _Report()
    tr = None
    arrays = None
    if trace:
        T = iters + 1
        arrays = {"support": np.zeros((T, s), np.int32), "kth": np.zeros((T, 2)),
                  "min_gap": np.zeros(T), "mu": np.zeros(T), "bt": np.zeros(T, np.int32),
                  "min_margin": np.zeros(T), "resid2": np.zeros(T),
                  "x": np.zeros((T, n)) if trace == "x" else None, "mu_fallback": np.zeros(T, np.int32),
                  "num": np.zeros(T), "xnorm2": np.zeros(T)}
        tr = _Trace(*[_ptr(arrays[f]) if arrays[f] is not None else None for f, _ in _Trace._fields_])
    ptrs = [(ctypes.c_void_p * (iters + 1))(*[_ptr(a) for a in lst]) for lst in (A1l, A2l, yl)]
    lib().qo_niht_seq(ptrs[0], ptrs[1], ptrs[2], m, n, s, iters, ctypes.byref(p), _ptr(x), _ptr(sup),
                      ctypes.byref(tr) if tr is not None else None, ctypes.byref(rep))
    if arrays is not None:
        T = rep.iters_run + 1
        arrays = {kk: vv[:T] for kk, vv in arrays.items() if vv is not None}
    return NihtResult(x=x, support=sup, status=rep.status, iters_run=rep.iters_run,
                      backtracks=rep.backtracks, support_changes=rep.support_changes,
                      resid_norm2=rep.resid_norm2, mu=rep.mu, trace=arrays)


def phi_stream(k: int) -> int:
    """Random-number stream of the k-th realization of Q(Phi) (k = 1, 2, ...): 0 and 1 for the
    first two (the fixed quantizations Q1, Q2), then 0x1000 + k."""
    return k - 1 if k <= 2 else 0x1000 + k


def y_stream(t: int) -> int:
    """Stream of the t-th realization of Q(y) (t = 1, 2, ...): 2 for the first, then 0x2000 + t."""
    return 2 if t == 1 else 0x2000 + t


def qiht_fresh(phi: np.ndarray, y: np.ndarray, s: int, iters: int, *, bits_phi: int, bits_y: int,
               seed: int, odd: bool = False, **kw):
    """Algorithm 2 as written: iteration t uses fresh realizations Phi-hat_{2t-1} (gradient),
    Phi-hat_{2t} (A2 x, step size, backtracking test) and y-hat_t; the initial support comes
    from Phi-hat_1 and y-hat_1. Realization k of Q(Phi) uses stream phi_stream(k), realization t
    of Q(y) stream y_stream(t); every realization of Phi shares the scale max |Phi|."""
    _, sphi = quantize(phi, bits_phi, seed, 0, odd=odd)
    _, sy = quantize(y, bits_y, seed, 2, odd=odd)

    def dphi(k):
        cds, _ = quantize(phi, bits_phi, seed, phi_stream(k), sphi, odd=odd)
        return dequantize(cds, bits_phi, sphi, odd=odd)

    def dy(t):
        cds, _ = quantize(y, bits_y, seed, y_stream(t), sy, odd=odd)
        return dequantize(cds, bits_y, sy, odd=odd)

    A1s = [dphi(1)] + [dphi(2 * t - 1) for t in range(1, iters + 1)]
    A2s = [dphi(2)] + [dphi(2 * t) for t in range(1, iters + 1)]
    ys = [dy(1)] + [dy(t) for t in range(1, iters + 1)]
    return niht_seq(A1s, A2s, ys, s, iters, **kw), {"scale_phi": sphi, "scale_y": sy}


def qiht(phi: np.ndarray, y: np.ndarray, s: int, iters: int, *, bits_phi: int, bits_y: int,
         seed: int, odd: bool = False, **kw):
    """Quantize Phi twice (streams 0 and 1) and y once (stream 2), then run Algorithm 2.
    odd=True quantizes all three on the odd grids of levels(bits, odd=True).

    Returns (NihtResult, dict with codes and scales)."""
    c1, sphi = quantize(phi, bits_phi, seed, 0, odd=odd)
    c2, _ = quantize(phi, bits_phi, seed, 1, sphi, odd=odd)
    cy, sy = quantize(y, bits_y, seed, 2, odd=odd)
    A1 = dequantize(c1, bits_phi, sphi, odd=odd)
    A2 = dequantize(c2, bits_phi, sphi, odd=odd)
    yq = dequantize(cy, bits_y, sy, odd=odd)
    res = niht(A1, A2, yq, s, iters, **kw)
    return res, {"codes1": c1, "codes2": c2, "codes_y": cy, "scale_phi": sphi, "scale_y": sy,
                 "A1": A1, "A2": A2, "yq": yq}
