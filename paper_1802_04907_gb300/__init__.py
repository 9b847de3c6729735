"""QIHT on GB300: thin Python binding of the C ABI in include/qiht.h.

Every step of the method runs in the CUDA library libqiht.so; this module only
marshals arguments (torch tensors for device memory, torch streams) and keeps
the names of the C entry points. There is no CPU fallback: if the library is
missing, every call raises.

Paper: Gurel et al., "Compressive Sensing Using Iterative Hard Thresholding with
Low Precision Data Representation" (IEEE TSP 2020), Algorithm 2 (QIHT) with the
stochastic quantizer of Section III-A.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqiht.so")

OK, ERR_ARG, ERR_BITS, ERR_NONFINITE, ERR_TIMEOUT, ERR_BACKTRACK_CAP, ERR_CUDA, ERR_WORKSPACE = range(8)
SCALE_GIVEN = 1
CHECK_FINITE = 2
ODD_LEVELS = 4
SOLVE_EAGER = 1
SOLVE_TEST_TIMEOUT = 2
SOLVE_FP8 = 4

# stream ids of the random numbers, by convention of the solver
STREAM_Q1, STREAM_Q2, STREAM_Y = 0, 1, 2


class QihtError(RuntimeError):
    def __init__(self, status: int, where: str):
        detail = ""
        if status == ERR_CUDA:
            try:
                detail = " [" + lib().qiht_last_error().decode() + "]"
            except Exception:
                pass
        super().__init__(f"{where}: {status_string(status)} ({status}){detail}")
        self.status = status


class _Codes(ctypes.Structure):
    _fields_ = [("words", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("rows", ctypes.c_int32),
                ("cols", ctypes.c_int32), ("bits", ctypes.c_int32), ("ld_words", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Problem(ctypes.Structure):
    _fields_ = [("Q1", _Codes), ("Q2", _Codes), ("y", _Codes), ("s", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("x", ctypes.c_void_p), ("support", ctypes.c_void_p), ("report", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("c", ctypes.c_double), ("max_backtrack", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("tol", ctypes.c_double), ("mu_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


MU_FORWARD_SQ, MU_CROSS = 0, 1


def _mu_mode(mode) -> int:
    """QIHT_MU_FORWARD_SQ for "forward" (the default) or QIHT_MU_CROSS for "cross"."""
    if mode in (MU_FORWARD_SQ, "forward", "forward_sq"):
        return MU_FORWARD_SQ
    if mode in (MU_CROSS, "cross"):
        return MU_CROSS
    raise ValueError(f"mu_mode {mode!r}")


class _Report(ctypes.Structure):
    _fields_ = [("iters_run", ctypes.c_int32), ("backtracks", ctypes.c_int32),
                ("support_changes", ctypes.c_int32), ("status", ctypes.c_int32),
                ("resid_norm2", ctypes.c_double), ("mu", ctypes.c_double),
                ("full_selects", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("phase_us", ctypes.c_float * 8)]


class _Trace(ctypes.Structure):
    _fields_ = [("support", ctypes.c_void_p), ("kth", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("bt", ctypes.c_void_p), ("resid2", ctypes.c_void_p)]


REPORT_BYTES = ctypes.sizeof(_Report)


class _FlyOp(ctypes.Structure):
    _fields_ = [("uv", ctypes.c_void_p), ("table", ctypes.c_void_p), ("baselines", ctypes.c_int32),
                ("grid", ctypes.c_int32)]


FLY_MAX_GRID = 256


class _SepOp(ctypes.Structure):
    _fields_ = [("factor", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("N", ctypes.c_int32), ("M", ctypes.c_int32)]


SEP_MAX_N = 512

EXPORTS = ["qiht_status_string", "qiht_abi_version", "qiht_last_error", "qiht_ld_words", "qiht_quantize",
           "qiht_quantize_pair",
           "qiht_gemv_t_workspace_size", "qiht_gemv_t", "qiht_gemv_t_prescaled",
           "qiht_gemv_cols_workspace_size", "qiht_gemv_cols", "qiht_gemv_cols_static",
           "qiht_top_s_workspace_size", "qiht_top_s", "qiht_solve_workspace_size", "qiht_niht_solve",
           "qiht_clear_graph_cache", "qiht_solve_batched_workspace_size", "qiht_niht_solve_batched",
           "qiht_gemv_t_multi_workspace_size", "qiht_gemv_t_multi", "qiht_gemv_t_multi_fp8",
           "qiht_solve_multi_workspace_size",
           "qiht_niht_solve_multi", "qiht_solve_fresh_workspace_size", "qiht_niht_solve_fresh",
           "qiht_unrolled_workspace_size", "qiht_unrolled_forward", "qiht_unrolled_backward",
           "qiht_fly_quantize", "qiht_gemv_t_fly", "qiht_niht_solve_fresh_fly",
           "qiht_solve_separable_workspace_size", "qiht_niht_solve_separable", "qiht_sep_quantize_factor",
           "qiht_sep_apply"]

_lib = None


def lib():
    """The loaded libqiht.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1802_04907_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, U32, U64, SZ = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_size_t)
        sig = {
            "qiht_status_string": ([I32], ctypes.c_char_p),
            "qiht_abi_version": ([], I32),
            "qiht_last_error": ([], ctypes.c_char_p),
            "qiht_ld_words": ([I32, I32], I32),
            "qiht_quantize": ([P, I32, I32, I64, I32, U64, U32, I32, P, I32, P, P], I32),
            "qiht_quantize_pair": ([P, I32, I32, I64, I32, U64, U32, U32, I32, P, P, I32, P, P], I32),
            "qiht_gemv_t_workspace_size": ([], SZ),
            "qiht_gemv_t": ([ctypes.POINTER(_Codes), P, P, P, SZ, P], I32),
            "qiht_gemv_t_prescaled": ([ctypes.POINTER(_Codes), P, P, P, P], I32),
            "qiht_gemv_cols_workspace_size": ([I32, I32], SZ),
            "qiht_gemv_cols": ([ctypes.POINTER(_Codes), P, P, I32, P, P, SZ, P], I32),
            "qiht_gemv_cols_static": ([ctypes.POINTER(_Codes), P, P, I32, P, P], I32),
            "qiht_top_s_workspace_size": ([I32], SZ),
            "qiht_top_s": ([P, I32, I32, P, P, P, P, SZ, P], I32),
            "qiht_solve_workspace_size": ([I32, I32, I32], SZ),
            "qiht_niht_solve": ([ctypes.POINTER(_Codes), ctypes.POINTER(_Codes), ctypes.POINTER(_Codes), I32, I32,
                                 ctypes.POINTER(_Params), P, P, P, ctypes.POINTER(_Trace), P, SZ, P], I32),
            "qiht_clear_graph_cache": ([], None),
            "qiht_solve_batched_workspace_size": ([I32], SZ),
            "qiht_niht_solve_batched": ([ctypes.POINTER(_Problem), I32, I32, ctypes.POINTER(_Params), P, SZ, P], I32),
            "qiht_gemv_t_multi_workspace_size": ([I32, I32], SZ),
            "qiht_gemv_t_multi": ([ctypes.POINTER(_Codes), P, I64, I32, P, I64, P, P, SZ, P], I32),
            "qiht_gemv_t_multi_fp8": ([ctypes.POINTER(_Codes), P, I64, I32, P, I64, P, P, SZ, P], I32),
            "qiht_solve_multi_workspace_size": ([I32, I32, I32, I32], SZ),
            "qiht_solve_fresh_workspace_size": ([I32, I32, I32, I32, I32], SZ),
            "qiht_unrolled_workspace_size": ([I32, I32, I32, I32, I32], SZ),
            "qiht_unrolled_forward": ([ctypes.POINTER(_Codes), ctypes.POINTER(_Codes), I32, P, P, P, I32, I32, P, P,
                                       SZ, P], I32),
            "qiht_unrolled_backward": ([ctypes.POINTER(_Codes), ctypes.POINTER(_Codes), I32, P, P, P, I32, I32, P, P,
                                        P, P, P, SZ, P], I32),
            "qiht_niht_solve_fresh": ([P, I64, P, I32, I32, I32, I32, U64, I32, I32, I32, ctypes.POINTER(_Params),
                                       P, P, P, ctypes.POINTER(_Trace), P, SZ, P], I32),
            "qiht_niht_solve_multi": ([ctypes.POINTER(_Codes), ctypes.POINTER(_Codes), ctypes.POINTER(_Codes), I32,
                                       I32, I32, ctypes.POINTER(_Params), P, P, P, P, SZ, P], I32),
            "qiht_fly_quantize": ([ctypes.POINTER(_FlyOp), I32, U64, U32, U32, I32, P, P, I32, P, P], I32),
            "qiht_gemv_t_fly": ([ctypes.POINTER(_FlyOp), I32, U64, U32, I32, P, P, P, P], I32),
            "qiht_niht_solve_fresh_fly": ([ctypes.POINTER(_FlyOp), P, I32, I32, U64, I32, I32, I32,
                                           ctypes.POINTER(_Params), P, P, P, ctypes.POINTER(_Trace), P, SZ, P], I32),
            "qiht_solve_separable_workspace_size": ([I32, I32, I32], SZ),
            "qiht_niht_solve_separable": ([ctypes.POINTER(_SepOp), P, I32, I32, U64, I32, I32, I32,
                                           ctypes.POINTER(_Params), P, P, P, ctypes.POINTER(_Trace), P, SZ, P], I32),
            "qiht_sep_quantize_factor": ([ctypes.POINTER(_SepOp), I32, U64, U32, I32, P, P, P, P], I32),
            "qiht_sep_apply": ([ctypes.POINTER(_SepOp), P, I32, P, P, P, SZ, P], I32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().qiht_status_string(status).decode()
    except Exception:
        return f"status {status}"


def _check(status: int, where: str):
    if status != OK:
        raise QihtError(status, where)


def _stream(stream, current=None) -> int:
    """Raw handle of the stream a call launches on (None: torch's current stream).

    When an explicit stream is not the current one, it is first made to wait for the
    current stream's queued work: the buffers a wrapper (or its caller) has just taken
    from torch's caching allocator come from the current stream's pool, and may be
    blocks that kernels queued there still read or write. `current` stands in for
    torch.cuda.current_stream() (tests)."""
    if stream is None:
        return (current if current is not None else torch.cuda.current_stream()).cuda_stream
    if hasattr(stream, "cuda_stream"):
        s = stream
    else:
        s = torch.cuda.ExternalStream(int(stream))
    cur = current if current is not None else torch.cuda.current_stream()
    if s.cuda_stream != cur.cuda_stream:
        s.wait_stream(cur)
    return s.cuda_stream


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _need(t, n: int, dtype, name: str) -> None:
    """The kernels take raw pointers: a vector of the wrong size or type would be read out of
    bounds, so the wrappers refuse it before any launch."""
    ok = isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() == n
    if not ok:
        got = (f"shape {tuple(t.shape)}, {t.dtype}, {'cuda' if t.is_cuda else 'cpu'}, contiguous={t.is_contiguous()}"
               if isinstance(t, torch.Tensor) else type(t).__name__)
        raise ValueError(f"{name}: needs a contiguous CUDA {dtype} tensor of {n} elements; got {got}")


def _hold(t: torch.Tensor, stream, current=None) -> None:
    """A buffer allocated here (a temporary or a new output) that work queued on `stream` uses:
    when that is not the current stream, tell torch's caching allocator, so that the memory
    is not handed out again before the work ends."""
    if stream is None:
        return
    s = stream if hasattr(stream, "cuda_stream") else torch.cuda.ExternalStream(int(stream))
    cur = current if current is not None else torch.cuda.current_stream(t.device)
    if s.cuda_stream != cur.cuda_stream:
        t.record_stream(s)


def _ws(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def ld_words(rows: int, bits: int) -> int:
    return int(lib().qiht_ld_words(rows, bits))


def odd_levels(bits: int) -> int:
    """Levels of the odd grid of b bits: 2^(b-1) + 1, spacing 1/2^(b-2) (0 is a level)."""
    return 2 ** (bits - 1) + 1


@dataclass
class Codes:
    """A quantized matrix (rows x cols) or vector (cols = 1) in the column-packed layout."""
    words: torch.Tensor      # int32 view of the u32 words, cols * ld_words
    scale: torch.Tensor      # float32 [1]: c = max |v|
    rows: int
    cols: int
    bits: int
    levels: int = 0          # 0 (= 2^bits, the default grid) or odd_levels(bits)

    @property
    def ld_words(self) -> int:
        return ld_words(self.rows, self.bits)

    @property
    def odd(self) -> bool:
        return self.levels == odd_levels(self.bits) and self.levels != 2**self.bits

    def c_struct(self) -> _Codes:
        """The C descriptor. The kernels read cols * ld_words words and one scale through raw
        pointers, so a hand-made or sliced Codes of the wrong size, type or device is refused."""
        w, sc = self.words, self.scale
        if self.bits not in (2, 4, 8) or self.rows < 1 or self.cols < 1:
            raise ValueError(f"Codes: bits {self.bits}, rows {self.rows}, cols {self.cols} out of range")
        need = self.cols * self.ld_words
        if not (isinstance(w, torch.Tensor) and w.is_cuda and w.dtype == torch.int32 and w.is_contiguous() and
                w.numel() == need):
            got = (f"shape {tuple(w.shape)}, {w.dtype}, {'cuda' if w.is_cuda else 'cpu'}" if isinstance(w, torch.Tensor)
                   else type(w).__name__)
            raise ValueError(f"Codes.words: needs a contiguous CUDA int32 tensor of cols * ld_words = {need} "
                             f"elements; got {got}")
        if not (isinstance(sc, torch.Tensor) and sc.is_cuda and sc.dtype == torch.float32 and sc.numel() >= 1 and
                sc.device == w.device):
            raise ValueError("Codes.scale: needs a CUDA float32 tensor (one element) on the device of the words")
        return _Codes(w.data_ptr(), sc.data_ptr(), self.rows, self.cols, self.bits, self.ld_words, self.levels, 0)

    @property
    def nbytes(self) -> int:
        return self.words.numel() * 4


def quantize(v: torch.Tensor, bits: int, seed: int, stream_id: int, *, scale: torch.Tensor | None = None,
             scale_given: bool = False, check_finite: bool = False, out: Codes | None = None,
             odd: bool = False, stream=None) -> Codes:
    """qiht_quantize: Q(v, b) of a float32 matrix (rows x cols, row-major) or vector.
    odd=True quantizes on the odd grid of odd_levels(bits) levels."""
    assert v.is_cuda and v.dtype == torch.float32
    if v.dim() == 1:
        rows, cols, ld = v.shape[0], 1, 1
    else:
        rows, cols = v.shape
        ld = v.stride(0)
        assert v.stride(1) == 1
    ldw = ld_words(rows, bits) if bits in (2, 4, 8) else 4
    if out is None:
        words = torch.empty(cols * ldw, dtype=torch.int32, device=v.device)
        sc = scale if scale is not None else torch.zeros(1, dtype=torch.float32, device=v.device)
        out = Codes(words, sc, rows, cols, bits)
    elif scale is not None:
        out.scale = scale
    out.levels = odd_levels(bits) if odd else 0
    flags = (SCALE_GIVEN if scale_given else 0) | (CHECK_FINITE if check_finite else 0) | (ODD_LEVELS if odd else 0)
    st = lib().qiht_quantize(v.data_ptr(), rows, cols, ld, bits, seed & (2**64 - 1), stream_id, flags,
                             out.words.data_ptr(), ldw, out.scale.data_ptr(), _stream(stream))
    _check(st, "qiht_quantize")
    _hold(out.words, stream)
    _hold(out.scale, stream)
    return out


def gemv_t(Q: Codes, r: torch.Tensor, g: torch.Tensor | None = None, *, workspace: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    """qiht_gemv_t: g = Q^T r."""
    _need(r, Q.rows, torch.float32, "r")
    if g is None:
        g = torch.empty(Q.cols, dtype=torch.float32, device=r.device)
    _need(g, Q.cols, torch.float32, "g")
    ws = workspace if workspace is not None else _ws(lib().qiht_gemv_t_workspace_size(), r.device)
    c = Q.c_struct()
    _check(lib().qiht_gemv_t(ctypes.byref(c), r.data_ptr(), g.data_ptr(), ws.data_ptr(), ws.numel(),
                             _stream(stream)), "qiht_gemv_t")
    if workspace is None:
        _hold(ws, stream)
    _hold(g, stream)
    return g


def gemv_t_multi(Q: Codes, R: torch.Tensor, G: torch.Tensor | None = None, *, status: torch.Tensor | None = None,
                 workspace: torch.Tensor | None = None, fp8: bool = False, stream=None) -> torch.Tensor:
    """qiht_gemv_t_multi (fp8: qiht_gemv_t_multi_fp8): G = Q^T R for the rows of R (nrhs x rows
    residuals) on the tensor cores."""
    if not (R.dim() == 2 and R.is_cuda and R.dtype == torch.float32 and R.stride(1) == 1 and R.shape[1] == Q.rows):
        raise ValueError(f"R: needs a CUDA float32 nrhs x {Q.rows} matrix with unit column stride; got "
                         f"shape {tuple(R.shape)}, {R.dtype}, strides {R.stride()}")
    nrhs = R.shape[0]
    if G is None:
        G = torch.empty((nrhs, Q.cols), dtype=torch.float32, device=R.device)
    if not (G.dim() == 2 and G.is_cuda and G.dtype == torch.float32 and G.stride(1) == 1 and
            tuple(G.shape) == (nrhs, Q.cols)):
        raise ValueError(f"G: needs a CUDA float32 {nrhs} x {Q.cols} matrix with unit column stride")
    ws = workspace if workspace is not None else _ws(lib().qiht_gemv_t_multi_workspace_size(Q.rows, nrhs), R.device)
    c = Q.c_struct()
    fn = lib().qiht_gemv_t_multi_fp8 if fp8 else lib().qiht_gemv_t_multi
    _check(fn(ctypes.byref(c), R.data_ptr(), R.stride(0), nrhs, G.data_ptr(), G.stride(0),
              status.data_ptr() if status is not None else None, ws.data_ptr(), ws.numel(), _stream(stream)),
           "qiht_gemv_t_multi_fp8" if fp8 else "qiht_gemv_t_multi")
    if workspace is None:
        _hold(ws, stream)
    _hold(G, stream)
    return G


def gemv_t_prescaled(Q: Codes, r: torch.Tensor, rmax: torch.Tensor, g: torch.Tensor, *, stream=None):
    """qiht_gemv_t_prescaled: g = Q^T r with max |r| given in rmax (one kernel launch)."""
    _need(r, Q.rows, torch.float32, "r")
    _need(rmax, 1, torch.float32, "rmax")
    _need(g, Q.cols, torch.float32, "g")
    c = Q.c_struct()
    _check(lib().qiht_gemv_t_prescaled(ctypes.byref(c), r.data_ptr(), rmax.data_ptr(), g.data_ptr(),
                                       _stream(stream)), "qiht_gemv_t_prescaled")
    return g


def gemv_cols(Q: Codes, cols: torch.Tensor, coef: torch.Tensor, z: torch.Tensor | None = None, *,
              workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """qiht_gemv_cols: z = Q[:, cols] coef."""
    count = cols.numel()
    _need(cols, count, torch.int32, "cols")
    _need(coef, count, torch.float32, "coef")
    if z is None:
        z = torch.empty(Q.rows, dtype=torch.float32, device=coef.device)
    _need(z, Q.rows, torch.float32, "z")
    ws = workspace if workspace is not None else _ws(lib().qiht_gemv_cols_workspace_size(Q.rows, count), coef.device)
    c = Q.c_struct()
    _check(lib().qiht_gemv_cols(ctypes.byref(c), cols.data_ptr(), coef.data_ptr(), count, z.data_ptr(),
                                ws.data_ptr(), ws.numel(), _stream(stream)), "qiht_gemv_cols")
    if workspace is None:
        _hold(ws, stream)
    _hold(z, stream)
    return z


def top_s(a: torch.Tensor, s: int, *, with_values: bool = True, stream=None):
    """qiht_top_s: H_s of a vector; returns (indices ascending, values, kth[2])."""
    n = a.numel()
    _need(a, n, torch.float32, "a")
    idx = torch.empty(s, dtype=torch.int32, device=a.device)
    val = torch.empty(s, dtype=torch.float32, device=a.device) if with_values else None
    kth = torch.empty(2, dtype=torch.float32, device=a.device)
    wsb = int(lib().qiht_top_s_workspace_size(n))
    ws = _ws(wsb, a.device) if wsb else None
    _check(lib().qiht_top_s(a.data_ptr(), n, s, idx.data_ptr(), _ptr(val), kth.data_ptr(), _ptr(ws),
                            ws.numel() if ws is not None else 0, _stream(stream)), "qiht_top_s")
    for t in (idx, val, kth, ws):
        if t is not None:
            _hold(t, stream)
    return idx, val, kth


def solve_workspace_size(m: int, n: int, s: int) -> int:
    return int(lib().qiht_solve_workspace_size(m, n, s))


@dataclass
class Report:
    iters_run: int
    backtracks: int
    support_changes: int
    status: int
    resid_norm2: float
    mu: float
    full_selects: int = 0
    phase_us: tuple = ()

    def __eq__(self, other):       # the diagnostic timings differ from run to run
        return (self.iters_run, self.backtracks, self.support_changes, self.status, self.resid_norm2, self.mu,
                self.full_selects) == (other.iters_run, other.backtracks, other.support_changes, other.status,
                                       other.resid_norm2, other.mu, other.full_selects)


def report_from_bytes(buf: bytes) -> Report:
    r = _Report.from_buffer_copy(buf)
    return Report(r.iters_run, r.backtracks, r.support_changes, r.status, r.resid_norm2, r.mu, r.full_selects,
                  tuple(float(v) for v in r.phase_us))


class Solver:
    """Buffers of one qiht_niht_solve configuration (outputs, workspace, trace).

    Keeping the same Solver object keeps the same pointers, so the library's
    cached CUDA graph is reused on every call."""

    def __init__(self, m: int, n: int, s: int, iters: int, *, device="cuda", trace: bool = False,
                 k: float = 2.0, c: float = 0.01, max_backtrack: int = 32, eager: bool = False,
                 test_timeout: bool = False, tol: float = 0.0, mu_mode="forward"):
        self.m, self.n, self.s, self.iters = m, n, s, iters
        self.params = _Params(k, c, max_backtrack,
                              (SOLVE_EAGER if eager else 0) | (SOLVE_TEST_TIMEOUT if test_timeout else 0),
                              float(tol), _mu_mode(mu_mode), 0)
        self.x = torch.empty(n, dtype=torch.float32, device=device)
        self.support = torch.empty(s, dtype=torch.int32, device=device)
        self.report = torch.zeros(REPORT_BYTES, dtype=torch.uint8, device=device)
        self.workspace = _ws(solve_workspace_size(m, n, s), device)
        self.trace = None
        if trace:
            T = iters + 1
            self.trace = {"support": torch.zeros((T, s), dtype=torch.int32, device=device),
                          "kth": torch.zeros((T, 2), dtype=torch.float32, device=device),
                          "mu": torch.zeros(T, dtype=torch.float64, device=device),
                          "bt": torch.zeros(T, dtype=torch.int32, device=device),
                          "resid2": torch.zeros(T, dtype=torch.float64, device=device)}

    def __call__(self, Q1: Codes, Q2: Codes, y: Codes, stream=None):
        """qiht_niht_solve (asynchronous); results in self.x, self.support, self.report."""
        c1, c2, cy = Q1.c_struct(), Q2.c_struct(), y.c_struct()
        tr = None
        if self.trace is not None:
            t = self.trace
            tr = _Trace(t["support"].data_ptr(), t["kth"].data_ptr(), t["mu"].data_ptr(), t["bt"].data_ptr(),
                        t["resid2"].data_ptr())
        st = lib().qiht_niht_solve(ctypes.byref(c1), ctypes.byref(c2), ctypes.byref(cy), self.s, self.iters,
                                   ctypes.byref(self.params), self.x.data_ptr(), self.support.data_ptr(),
                                   self.report.data_ptr(), ctypes.byref(tr) if tr is not None else None,
                                   self.workspace.data_ptr(), self.workspace.numel(), _stream(stream))
        _check(st, "qiht_niht_solve")
        for t in self._buffers():
            _hold(t, stream)
        return self

    def _buffers(self):
        yield from (self.x, self.support, self.report, self.workspace)
        if self.trace is not None:
            yield from self.trace.values()

    def read_report(self) -> Report:
        return report_from_bytes(bytes(self.report.cpu().numpy().tobytes()))


def niht_solve(Q1: Codes, Q2: Codes, y: Codes, s: int, iters: int, *, trace: bool = False, stream=None, **kw):
    """One QIHT solve (Algorithm 2). Returns the Solver holding x, support, report (and trace)."""
    sv = Solver(Q1.rows, Q1.cols, s, iters, device=Q1.words.device, trace=trace, **kw)
    return sv(Q1, Q2, y, stream=stream)


def niht_solve_fresh(phi: torch.Tensor, y: torch.Tensor, bits_phi: int, bits_y: int, seed: int, s: int, iters: int,
                     *, odd: bool = False, trace: bool = False, k: float = 2.0, c: float = 0.01,
                     max_backtrack: int = 32, tol: float = 0.0, mu_mode="forward", stream=None) -> Solver:
    """qiht_niht_solve_fresh: Algorithm 2 with new quantizations of Phi and y in every iteration.
    Returns a Solver-like object holding x, support, report (and trace)."""
    if not (isinstance(phi, torch.Tensor) and phi.is_cuda and phi.dtype == torch.float32 and phi.dim() == 2 and
            phi.stride(1) == 1):
        raise ValueError("phi: needs a CUDA float32 m x n matrix with unit column stride")
    m, n = phi.shape
    _need(y, m, torch.float32, "y")
    sv = Solver(m, n, s, iters, device=phi.device, trace=trace, k=k, c=c, max_backtrack=max_backtrack, tol=tol,
                mu_mode=mu_mode)
    ws = _ws(lib().qiht_solve_fresh_workspace_size(m, n, s, bits_phi, bits_y), phi.device)
    tr = None
    if sv.trace is not None:
        t = sv.trace
        tr = _Trace(t["support"].data_ptr(), t["kth"].data_ptr(), t["mu"].data_ptr(), t["bt"].data_ptr(),
                    t["resid2"].data_ptr())
    st = lib().qiht_niht_solve_fresh(phi.data_ptr(), phi.stride(0), y.data_ptr(), m, n, bits_phi, bits_y,
                                     seed & (2**64 - 1), ODD_LEVELS if odd else 0, s, iters, ctypes.byref(sv.params),
                                     sv.x.data_ptr(), sv.support.data_ptr(), sv.report.data_ptr(),
                                     ctypes.byref(tr) if tr is not None else None, ws.data_ptr(), ws.numel(),
                                     _stream(stream))
    _check(st, "qiht_niht_solve_fresh")
    sv.workspace = ws
    return sv


class FlyOp:
    """The gridded interferometry operator of qiht_fly_op: Phi[k][p] = table[t_kp] and
    Phi[K + k][p] = table[g + t_kp], t_kp = (u_k (ix - g/2) + v_k (iy - g/2)) mod g, p = ix g + iy.
    uv: CUDA int32 (K, 2); table: CUDA float32 (2g,). Holds both tensors for the calls that use it."""

    def __init__(self, uv: torch.Tensor, table: torch.Tensor, grid: int):
        if not (uv.is_cuda and uv.dtype == torch.int32 and uv.dim() == 2 and uv.shape[1] == 2 and uv.is_contiguous()):
            raise ValueError("uv: needs a contiguous CUDA int32 (K, 2) tensor")
        _need(table, 2 * grid, torch.float32, "table")
        self.uv, self.table, self.grid = uv, table, int(grid)
        self.baselines = int(uv.shape[0])
        self.rows, self.cols = 2 * self.baselines, self.grid * self.grid

    def c_struct(self) -> _FlyOp:
        return _FlyOp(self.uv.data_ptr(), self.table.data_ptr(), self.baselines, self.grid)


def fly_quantize(op: FlyOp, bits: int, seed: int, stream_id: int, stream_b: int | None = None, *,
                 odd: bool = False, stream=None):
    """qiht_fly_quantize: the codes of the operator's Phi (one quantization, or two with stream_b)."""
    dev = op.uv.device
    ldw = ld_words(op.rows, bits)
    levels = odd_levels(bits) if odd else 2**bits
    scale = torch.empty(1, dtype=torch.float32, device=dev)
    wa = torch.empty((op.cols, ldw), dtype=torch.int32, device=dev)
    wb = torch.empty((op.cols, ldw), dtype=torch.int32, device=dev) if stream_b is not None else None
    c = op.c_struct()
    _check(lib().qiht_fly_quantize(ctypes.byref(c), bits, seed & (2**64 - 1), stream_id,
                                   stream_b if stream_b is not None else 0, ODD_LEVELS if odd else 0, wa.data_ptr(),
                                   wb.data_ptr() if wb is not None else None, ldw, scale.data_ptr(), _stream(stream)),
           "qiht_fly_quantize")
    for t in (wa, wb, scale):
        if t is not None:
            _hold(t, stream)
    qa = Codes(wa, scale, op.rows, op.cols, bits, levels)
    if wb is None:
        return qa
    return qa, Codes(wb, scale, op.rows, op.cols, bits, levels)


def gemv_t_fly(op: FlyOp, bits: int, seed: int, stream_id: int, r: torch.Tensor, g: torch.Tensor | None = None, *,
               odd: bool = False, scale: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """qiht_gemv_t_fly: g = Q^T r with Q generated and quantized inside the product."""
    _need(r, op.rows, torch.float32, "r")
    if g is None:
        g = torch.empty(op.cols, dtype=torch.float32, device=r.device)
    _need(g, op.cols, torch.float32, "g")
    if scale is None:
        scale = torch.empty(1, dtype=torch.float32, device=r.device)
    c = op.c_struct()
    _check(lib().qiht_gemv_t_fly(ctypes.byref(c), bits, seed & (2**64 - 1), stream_id, ODD_LEVELS if odd else 0,
                                 r.data_ptr(), g.data_ptr(), scale.data_ptr(), _stream(stream)), "qiht_gemv_t_fly")
    _hold(g, stream)
    _hold(scale, stream)
    return g


def niht_solve_fresh_fly(op: FlyOp, y: torch.Tensor, bits_phi: int, bits_y: int, seed: int, s: int, iters: int, *,
                         odd: bool = False, trace: bool = False, k: float = 2.0, c: float = 0.01,
                         max_backtrack: int = 32, tol: float = 0.0, mu_mode="forward", stream=None) -> Solver:
    """qiht_niht_solve_fresh_fly: Algorithm 2 with new realizations every iteration, Phi from the operator."""
    m, n = op.rows, op.cols
    _need(y, m, torch.float32, "y")
    sv = Solver(m, n, s, iters, device=y.device, trace=trace, k=k, c=c, max_backtrack=max_backtrack, tol=tol,
                mu_mode=mu_mode)
    ws = _ws(lib().qiht_solve_fresh_workspace_size(m, n, s, bits_phi, bits_y), y.device)
    tr = None
    if sv.trace is not None:
        t = sv.trace
        tr = _Trace(t["support"].data_ptr(), t["kth"].data_ptr(), t["mu"].data_ptr(), t["bt"].data_ptr(),
                    t["resid2"].data_ptr())
    cs = op.c_struct()
    st = lib().qiht_niht_solve_fresh_fly(ctypes.byref(cs), y.data_ptr(), bits_phi, bits_y, seed & (2**64 - 1),
                                         ODD_LEVELS if odd else 0, s, iters, ctypes.byref(sv.params), sv.x.data_ptr(),
                                         sv.support.data_ptr(), sv.report.data_ptr(),
                                         ctypes.byref(tr) if tr is not None else None, ws.data_ptr(), ws.numel(),
                                         _stream(stream))
    _check(st, "qiht_niht_solve_fresh_fly")
    sv.workspace = ws
    return sv


class SepOp:
    """The separable operator of qiht_sep_op: Phi = S (A (x) A) stacked real, with the factor
    given as the stacked real matrix [Re A; Im A] (CUDA float32, 2N x N) and the sampled
    positions k1 * N + k2 (CUDA int32, M)."""

    def __init__(self, factor: torch.Tensor, mask: torch.Tensor):
        if not (factor.is_cuda and factor.dtype == torch.float32 and factor.dim() == 2 and factor.is_contiguous()
                and factor.shape[0] == 2 * factor.shape[1]):
            raise ValueError("factor: needs a contiguous CUDA float32 2N x N tensor")
        if not (mask.is_cuda and mask.dtype == torch.int32 and mask.dim() == 1 and mask.is_contiguous()):
            raise ValueError("mask: needs a contiguous CUDA int32 vector")
        self.factor, self.mask = factor, mask
        self.N, self.M = int(factor.shape[1]), int(mask.shape[0])
        self.rows, self.cols = 2 * self.M, self.N * self.N

    def c_struct(self) -> _SepOp:
        return _SepOp(self.factor.data_ptr(), self.mask.data_ptr(), self.N, self.M)


def sep_quantize_factor(op: SepOp, bits: int, seed: int, stream_id: int, *, odd: bool = False, stream=None):
    """qiht_sep_quantize_factor: (codes uint16 as int16 tensor, dequantized factor, scale) of one
    quantization of the stacked factor."""
    dev = op.factor.device
    codes = torch.empty((2 * op.N, op.N), dtype=torch.int16, device=dev)
    fh = torch.empty((2 * op.N, op.N), dtype=torch.float32, device=dev)
    scale = torch.empty(1, dtype=torch.float32, device=dev)
    c = op.c_struct()
    _check(lib().qiht_sep_quantize_factor(ctypes.byref(c), bits, seed & (2**64 - 1), stream_id, ODD_LEVELS if odd else 0,
                                          codes.data_ptr(), fh.data_ptr(), scale.data_ptr(), _stream(stream)),
           "qiht_sep_quantize_factor")
    for t in (codes, fh, scale):
        _hold(t, stream)
    return codes, fh, scale


def sep_apply(op: SepOp, factor_hat: torch.Tensor, v: torch.Tensor, *, adjoint: bool = False, stream=None):
    """qiht_sep_apply: Phi-hat v (v of N^2 floats -> 2M) or, adjoint, Phi-hat^T v (2M -> N^2)."""
    _need(v, op.rows if adjoint else op.cols, torch.float32, "v")
    out = torch.empty(op.cols if adjoint else op.rows, dtype=torch.float32, device=v.device)
    ws = _ws(lib().qiht_solve_separable_workspace_size(op.N, op.M, 1), v.device)
    c = op.c_struct()
    _check(lib().qiht_sep_apply(ctypes.byref(c), factor_hat.data_ptr(), 1 if adjoint else 0, v.data_ptr(),
                                out.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)), "qiht_sep_apply")
    _hold(ws, stream)
    _hold(out, stream)
    return out


def niht_solve_separable(op: SepOp, y: torch.Tensor, bits_factor: int, bits_y: int, seed: int, s: int, iters: int, *,
                         odd: bool = False, trace: bool = False, k: float = 2.0, c: float = 0.01,
                         max_backtrack: int = 32, tol: float = 0.0, stream=None) -> Solver:
    """qiht_niht_solve_separable: Algorithm 2 on the separable operator with quantized factors."""
    m, n = op.rows, op.cols
    _need(y, m, torch.float32, "y")
    sv = Solver(m, n, s, iters, device=y.device, trace=trace, k=k, c=c, max_backtrack=max_backtrack, tol=tol)
    ws = _ws(lib().qiht_solve_separable_workspace_size(op.N, op.M, s), y.device)
    tr = None
    if sv.trace is not None:
        t = sv.trace
        tr = _Trace(t["support"].data_ptr(), t["kth"].data_ptr(), t["mu"].data_ptr(), t["bt"].data_ptr(),
                    t["resid2"].data_ptr())
    cs = op.c_struct()
    st = lib().qiht_niht_solve_separable(ctypes.byref(cs), y.data_ptr(), bits_factor, bits_y, seed & (2**64 - 1),
                                         ODD_LEVELS if odd else 0, s, iters, ctypes.byref(sv.params), sv.x.data_ptr(),
                                         sv.support.data_ptr(), sv.report.data_ptr(),
                                         ctypes.byref(tr) if tr is not None else None, ws.data_ptr(), ws.numel(),
                                         _stream(stream))
    _check(st, "qiht_niht_solve_separable")
    sv.workspace = ws
    return sv


class Unrolled:
    """K unrolled QIHT iterations (frozen support masks, no backtracking test) for nprob problems
    sharing m, n, bits: qiht_unrolled_forward / qiht_unrolled_backward with one workspace (the
    forward keeps the sqrt(K) checkpoints the backward recomputes from)."""

    def __init__(self, Q1s: list, Q2s: list, s: int, K: int):
        self.Q1s, self.Q2s, self.s, self.K = Q1s, Q2s, s, K
        self.P = len(Q1s)
        self.m, self.n = Q1s[0].rows, Q1s[0].cols
        dev = Q1s[0].words.device
        self.c1 = (_Codes * self.P)(*[q.c_struct() for q in Q1s])
        self.c2 = (_Codes * self.P)(*[q.c_struct() for q in Q2s])
        self.ws = _ws(lib().qiht_unrolled_workspace_size(self.P, self.m, self.n, s, K), dev)
        self.generation = 0   # forward() calls so far: the checkpoints are those of the latest one

    def forward(self, y: torch.Tensor, gre: torch.Tensor, gim: torch.Tensor, stream=None) -> torch.Tensor:
        """x_K for every problem (P x n) from y (P x 2m) and the gains (P x m each)."""
        _need(y, self.P * 2 * self.m, torch.float32, "y")
        _need(gre, self.P * self.m, torch.float32, "gain (real parts)")
        _need(gim, self.P * self.m, torch.float32, "gain (imaginary parts)")
        X = torch.empty(self.P, self.n, dtype=torch.float32, device=y.device)
        _check(lib().qiht_unrolled_forward(self.c1, self.c2, self.P, y.data_ptr(), gre.data_ptr(), gim.data_ptr(),
                                           self.s, self.K, X.data_ptr(), self.ws.data_ptr(), self.ws.numel(),
                                           _stream(stream)), "qiht_unrolled_forward")
        self.generation += 1
        return X

    def backward(self, y: torch.Tensor, gre: torch.Tensor, gim: torch.Tensor, Xbar: torch.Tensor, stream=None):
        """(dL/dy, dL/dRe g, dL/dIm g) from dL/dx_K, after forward() on the same inputs."""
        _need(y, self.P * 2 * self.m, torch.float32, "y")
        _need(gre, self.P * self.m, torch.float32, "gain (real parts)")
        _need(gim, self.P * self.m, torch.float32, "gain (imaginary parts)")
        Xbar = Xbar.contiguous()
        _need(Xbar, self.P * self.n, torch.float32, "Xbar")
        yb = torch.empty_like(y)
        ab = torch.empty_like(gre)
        bb = torch.empty_like(gim)
        _check(lib().qiht_unrolled_backward(self.c1, self.c2, self.P, y.data_ptr(), gre.data_ptr(), gim.data_ptr(),
                                            self.s, self.K, Xbar.contiguous().data_ptr(), yb.data_ptr(),
                                            ab.data_ptr(), bb.data_ptr(), self.ws.data_ptr(), self.ws.numel(),
                                            _stream(stream)), "qiht_unrolled_backward")
        return yb, ab, bb


class UnrolledQIHT(torch.autograd.Function):
    """x_K = unrolled QIHT(y, gain) with the hand-written adjoint as its backward."""

    @staticmethod
    def forward(ctx, y, gre, gim, op):
        y, gre, gim = y.contiguous(), gre.contiguous(), gim.contiguous()
        X = op.forward(y, gre, gim)
        ctx.op = op
        ctx.generation = op.generation
        ctx.save_for_backward(y, gre, gim)
        return X

    @staticmethod
    def backward(ctx, grad_x):
        y, gre, gim = ctx.saved_tensors
        if ctx.op.generation != ctx.generation:
            # another forward through the same op replaced the checkpoints: recompute this one's
            ctx.op.forward(y, gre, gim)
        yb, ab, bb = ctx.op.backward(y, gre, gim, grad_x)
        return yb, ab, bb, None


def unrolled_qiht(y: torch.Tensor, gre: torch.Tensor, gim: torch.Tensor, op: Unrolled) -> torch.Tensor:
    """Differentiable x_K (P x n) of the unrolled iterations in y (P x 2m) and the gain (P x m, P x m)."""
    return UnrolledQIHT.apply(y, gre, gim, op)


BATCH_MAX_ROWS, BATCH_MAX_COLS, BATCH_MAX_S = 2048, 8192, 256


class BatchResult:
    """Outputs of qiht_niht_solve_batched: x[i] (n_i), support[i] (s_i), report(i)."""

    def __init__(self, xs, sups, reports, workspace):
        self.x, self.support, self.reports, self.workspace = xs, sups, reports, workspace

    def report(self, i: int) -> Report:
        return report_from_bytes(bytes(self.reports[i].cpu().numpy().tobytes()))

    def all_reports(self) -> list:
        host = self.reports.cpu().numpy()
        return [report_from_bytes(bytes(host[i].tobytes())) for i in range(host.shape[0])]


def niht_solve_batched(problems: list, iters: int, *, k: float = 2.0, c: float = 0.01, max_backtrack: int = 32,
                       stream=None) -> BatchResult:
    """qiht_niht_solve_batched: problems is a list of (Q1, Q2, y, s) with Codes Q1, Q2, y."""
    nprob = len(problems)
    dev = problems[0][0].words.device
    xs = [torch.empty(pr[0].cols, dtype=torch.float32, device=dev) for pr in problems]
    sups = [torch.empty(pr[3], dtype=torch.int32, device=dev) for pr in problems]
    reports = torch.zeros((nprob, REPORT_BYTES), dtype=torch.uint8, device=dev)
    arr = (_Problem * nprob)()
    for i, (q1, q2, qy, s) in enumerate(problems):
        arr[i] = _Problem(q1.c_struct(), q2.c_struct(), qy.c_struct(), int(s), 0, xs[i].data_ptr(),
                          sups[i].data_ptr(), reports[i].data_ptr())
    ws = _ws(lib().qiht_solve_batched_workspace_size(nprob), dev)
    params = _Params(k, c, max_backtrack, 0, 0.0, MU_FORWARD_SQ, 0)
    st = lib().qiht_niht_solve_batched(arr, nprob, iters, ctypes.byref(params), ws.data_ptr(), ws.numel(),
                                       _stream(stream))
    _check(st, "qiht_niht_solve_batched")
    return BatchResult(xs, sups, reports, ws)


MULTI_MAX_ROWS, MULTI_MAX_COLS, MULTI_MAX_S = 16384, 32768, 256


class MultiResult:
    """Outputs of qiht_niht_solve_multi: x (nrhs x n), support (nrhs x s), report(k)."""

    def __init__(self, x, support, reports, workspace):
        self.x, self.support, self.reports, self.workspace = x, support, reports, workspace

    def report(self, k: int) -> Report:
        return report_from_bytes(bytes(self.reports[k].cpu().numpy().tobytes()))

    def all_reports(self) -> list:
        host = self.reports.cpu().numpy()
        return [report_from_bytes(bytes(host[i].tobytes())) for i in range(host.shape[0])]


def niht_solve_multi(Q1: Codes, Q2: Codes, ys: list, s: int, iters: int, *, k: float = 2.0, c: float = 0.01,
                     max_backtrack: int = 32, workspace: torch.Tensor | None = None, out: tuple | None = None,
                     fp8: bool = False, stream=None) -> MultiResult:
    """qiht_niht_solve_multi: Algorithm 2 for every observation in ys (Codes vectors) sharing Q1, Q2."""
    nrhs = len(ys)
    dev = Q1.words.device
    if out is None:
        X = torch.empty((nrhs, Q1.cols), dtype=torch.float32, device=dev)
        sup = torch.empty((nrhs, s), dtype=torch.int32, device=dev)
        reports = torch.zeros((nrhs, REPORT_BYTES), dtype=torch.uint8, device=dev)
    else:
        X, sup, reports = out
    ws = workspace if workspace is not None else _ws(lib().qiht_solve_multi_workspace_size(Q1.rows, Q1.cols, s,
                                                                                          nrhs), dev)
    arr = (_Codes * nrhs)(*[y.c_struct() for y in ys])
    c1, c2 = Q1.c_struct(), Q2.c_struct()
    params = _Params(k, c, max_backtrack, SOLVE_FP8 if fp8 else 0, 0.0, MU_FORWARD_SQ, 0)
    st = lib().qiht_niht_solve_multi(ctypes.byref(c1), ctypes.byref(c2), arr, nrhs, s, iters, ctypes.byref(params),
                                     X.data_ptr(), sup.data_ptr(), reports.data_ptr(), ws.data_ptr(), ws.numel(),
                                     _stream(stream))
    _check(st, "qiht_niht_solve_multi")
    return MultiResult(X, sup, reports, ws)


def quantize_pair(v: torch.Tensor, bits: int, seed: int, stream_a: int, stream_b: int, *,
                  out: tuple | None = None, odd: bool = False, stream=None) -> tuple:
    """qiht_quantize_pair: two independent quantizations of one matrix in one pass (shared scale)."""
    assert v.is_cuda and v.dtype == torch.float32 and v.dim() == 2 and v.stride(1) == 1
    rows, cols = v.shape
    ld = v.stride(0)
    ldw = ld_words(rows, bits) if bits in (2, 4, 8) else 4
    if out is None:
        sc = torch.zeros(1, dtype=torch.float32, device=v.device)
        out = (Codes(torch.empty(cols * ldw, dtype=torch.int32, device=v.device), sc, rows, cols, bits),
               Codes(torch.empty(cols * ldw, dtype=torch.int32, device=v.device), sc, rows, cols, bits))
    qa, qb = out
    qa.levels = qb.levels = odd_levels(bits) if odd else 0
    st = lib().qiht_quantize_pair(v.data_ptr(), rows, cols, ld, bits, seed & (2**64 - 1), stream_a, stream_b,
                                  ODD_LEVELS if odd else 0,
                                  qa.words.data_ptr(), qb.words.data_ptr(), ldw, qa.scale.data_ptr(),
                                  _stream(stream))
    _check(st, "qiht_quantize_pair")
    qb.scale = qa.scale
    for t in (qa.words, qb.words, qa.scale):
        _hold(t, stream)
    return qa, qb


def quantize_problem(phi: torch.Tensor, y: torch.Tensor, bits_phi: int, bits_y: int, seed: int, *,
                     out: tuple | None = None, odd: bool = False, stream=None):
    """Q1, Q2 (two independent quantizations of Phi, sharing its scale, in one pass) and Q(y);
    odd=True puts all three on the odd grids."""
    if out is None:
        q1, q2 = quantize_pair(phi, bits_phi, seed, STREAM_Q1, STREAM_Q2, odd=odd, stream=stream)
        qy = quantize(y, bits_y, seed, STREAM_Y, odd=odd, stream=stream)
        return q1, q2, qy
    q1, q2, qy = out
    quantize_pair(phi, bits_phi, seed, STREAM_Q1, STREAM_Q2, out=(q1, q2), odd=odd, stream=stream)
    quantize(y, bits_y, seed, STREAM_Y, out=qy, odd=odd, stream=stream)
    return q1, q2, qy


def clear_graph_cache():
    lib().qiht_clear_graph_cache()
