"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/qiht.h. Only host-side paths are called here (argument
checks that return before any CUDA call), so this runs without a GPU."""
import ctypes
import os
import re

import pytest

import paper_1802_04907_gb300 as q
from paper_1802_04907_gb300 import build as qbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qiht.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qiht_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return q.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "qiht_niht_solve" in names and "qiht_quantize" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(q.EXPORTS) == set(names)


def test_host_only_entry_points(lib):
    assert lib.qiht_abi_version() == 4
    assert q.status_string(q.OK) == "QIHT_OK"
    assert q.status_string(q.ERR_BACKTRACK_CAP) == "QIHT_ERR_BACKTRACK_CAP"
    # words per column: ceil(rows / (32/bits)) rounded up to a multiple of 4
    assert q.ld_words(8192, 8) == 2048 and q.ld_words(8192, 4) == 1024 and q.ld_words(8192, 2) == 512
    assert q.ld_words(4512, 2) == 284 and q.ld_words(1, 8) == 4 and q.ld_words(17, 2) == 4
    assert q.ld_words(10, 3) == -1 and q.ld_words(0, 8) == -1
    assert q.solve_workspace_size(8192, 32768, 256) > 0
    assert q.solve_workspace_size(0, 1, 1) == 0
    assert lib.qiht_gemv_t_workspace_size() >= 4


def test_argument_errors_return_before_launch(lib):
    P = ctypes.c_void_p
    # bits not in {2,4,8}
    assert lib.qiht_quantize(P(16), 4, 4, 4, 3, 0, 0, 0, P(16), 4, P(16), None) == q.ERR_BITS
    # null input
    assert lib.qiht_quantize(None, 4, 4, 4, 8, 0, 0, 0, P(16), 4, P(16), None) == q.ERR_ARG
    # wrong ld_words
    assert lib.qiht_quantize(P(16), 4, 4, 4, 8, 0, 0, 0, P(16), 5, P(16), None) == q.ERR_ARG
    # unknown flag
    assert lib.qiht_quantize(P(16), 4, 4, 4, 8, 0, 0, 64, P(16), 4, P(16), None) == q.ERR_ARG
    c = q._Codes(16, 16, 64, 128, 8, q.ld_words(64, 8))
    cy = q._Codes(16, 16, 64, 1, 8, q.ld_words(64, 8))
    prm = q._Params(2.0, 0.01, 32, 0)
    solve = lib.qiht_niht_solve
    # s > m, s < 1, null outputs, bad params, mismatched shapes, missing workspace
    assert solve(ctypes.byref(c), ctypes.byref(c), ctypes.byref(cy), 65, 10, ctypes.byref(prm), P(16), P(16),
                 P(16), None, P(256), 1 << 30, None) == q.ERR_ARG
    assert solve(ctypes.byref(c), ctypes.byref(c), ctypes.byref(cy), 0, 10, ctypes.byref(prm), P(16), P(16),
                 P(16), None, P(256), 1 << 30, None) == q.ERR_ARG
    assert solve(ctypes.byref(c), ctypes.byref(c), ctypes.byref(cy), 4, 10, ctypes.byref(prm), None, P(16),
                 P(16), None, P(256), 1 << 30, None) == q.ERR_ARG
    bad = q._Params(1.0, 0.01, 32, 0)     # k (1 - c) must exceed 1
    assert solve(ctypes.byref(c), ctypes.byref(c), ctypes.byref(cy), 4, 10, ctypes.byref(bad), P(16), P(16),
                 P(16), None, P(256), 1 << 30, None) == q.ERR_ARG
    c2 = q._Codes(16, 16, 64, 127, 8, q.ld_words(64, 8))
    assert solve(ctypes.byref(c), ctypes.byref(c2), ctypes.byref(cy), 4, 10, ctypes.byref(prm), P(16), P(16),
                 P(16), None, P(256), 1 << 30, None) == q.ERR_ARG
    assert solve(ctypes.byref(c), ctypes.byref(c), ctypes.byref(cy), 4, 10, ctypes.byref(prm), P(16), P(16),
                 P(16), None, None, 0, None) == q.ERR_WORKSPACE
    assert solve(ctypes.byref(c), ctypes.byref(c), ctypes.byref(cy), 4, 10, ctypes.byref(prm), P(16), P(16),
                 P(16), None, P(272), 1 << 30, None) == q.ERR_WORKSPACE      # not 256-byte aligned
    # the step-size mode and the residual tolerance: unknown mode, negative or non-finite tol,
    # the cross product across two grids
    for bad_p in (q._Params(2.0, 0.01, 32, 0, 0.0, 2, 0), q._Params(2.0, 0.01, 32, 0, -1.0, 0, 0),
                  q._Params(2.0, 0.01, 32, 0, float("nan"), 0, 0), q._Params(2.0, 0.01, 32, 0, float("inf"), 1, 0)):
        assert solve(ctypes.byref(c), ctypes.byref(c), ctypes.byref(cy), 4, 10, ctypes.byref(bad_p), P(16), P(16),
                     P(16), None, P(256), 1 << 30, None) == q.ERR_ARG
    c_odd = q._Codes(16, 16, 64, 128, 8, q.ld_words(64, 8), q.odd_levels(8))
    cross = q._Params(2.0, 0.01, 32, 0, 0.0, q.MU_CROSS, 0)
    assert solve(ctypes.byref(c), ctypes.byref(c_odd), ctypes.byref(cy), 4, 10, ctypes.byref(cross), P(16), P(16),
                 P(16), None, P(256), 1 << 30, None) == q.ERR_ARG
    # the batched and many-right-hand-side solvers take the defaults only
    pbt = q._Problem(c, c, cy, 4, 0, 16, 16, 16)
    for nd in (q._Params(2.0, 0.01, 32, 0, 1e-3, 0, 0), cross):
        assert lib.qiht_niht_solve_batched((q._Problem * 1)(pbt), 1, 5, ctypes.byref(nd), P(256), 1 << 20,
                                           None) == q.ERR_ARG
        assert lib.qiht_niht_solve_multi(ctypes.byref(c), ctypes.byref(c), (q._Codes * 1)(cy), 1, 4, 10,
                                         ctypes.byref(nd), P(16), P(16), P(16), P(256), 1 << 30, None) == q.ERR_ARG
    # m above the GEMV^T limit
    big = q._Codes(16, 16, 20000, 128, 8, q.ld_words(20000, 8))
    bigy = q._Codes(16, 16, 20000, 1, 8, q.ld_words(20000, 8))
    assert solve(ctypes.byref(big), ctypes.byref(big), ctypes.byref(bigy), 4, 10, ctypes.byref(prm), P(16),
                 P(16), P(16), None, P(256), 1 << 40, None) == q.ERR_ARG
    # top_s: s > n
    assert lib.qiht_top_s(P(16), 10, 11, P(16), None, None, None, 0, None) == q.ERR_ARG
    # past one CTA's keys the select needs its workspace
    assert lib.qiht_top_s_workspace_size(49152) == 0 and lib.qiht_top_s_workspace_size(49153) > 4 * 49153
    assert lib.qiht_top_s(P(16), 49153, 10, P(16), None, None, None, 0, None) == q.ERR_WORKSPACE
    assert lib.qiht_top_s(P(16), (1 << 24) + 1, 10, P(16), None, None, P(256), 1 << 30, None) == q.ERR_ARG
    # batched: empty batch, a problem above the limits, mixed widths, null outputs, no workspace
    assert lib.qiht_solve_batched_workspace_size(0) == 0 and lib.qiht_solve_batched_workspace_size(3) > 0
    pb = q._Problem(c, c, cy, 4, 0, 16, 16, 16)
    arr = (q._Problem * 1)(pb)
    assert lib.qiht_niht_solve_batched(arr, 0, 5, ctypes.byref(prm), P(256), 1 << 20, None) == q.ERR_ARG
    cbig = q._Codes(16, 16, q.BATCH_MAX_ROWS + 4, 8, 8, q.ld_words(q.BATCH_MAX_ROWS + 4, 8))
    cbigy = q._Codes(16, 16, q.BATCH_MAX_ROWS + 4, 1, 8, q.ld_words(q.BATCH_MAX_ROWS + 4, 8))
    arr2 = (q._Problem * 2)(pb, q._Problem(cbig, cbig, cbigy, 4, 0, 16, 16, 16))
    assert lib.qiht_niht_solve_batched(arr2, 2, 5, ctypes.byref(prm), P(256), 1 << 20, None) == q.ERR_ARG
    c4 = q._Codes(16, 16, 64, 128, 4, q.ld_words(64, 4))
    arr3 = (q._Problem * 2)(pb, q._Problem(c4, c4, cy, 4, 0, 16, 16, 16))
    assert lib.qiht_niht_solve_batched(arr3, 2, 5, ctypes.byref(prm), P(256), 1 << 20, None) == q.ERR_ARG
    arr4 = (q._Problem * 1)(q._Problem(c, c, cy, 4, 0, 16, 0, 16))
    assert lib.qiht_niht_solve_batched(arr4, 1, 5, ctypes.byref(prm), P(256), 1 << 20, None) == q.ERR_ARG
    assert lib.qiht_niht_solve_batched(arr, 1, 5, ctypes.byref(prm), None, 0, None) == q.ERR_WORKSPACE


def test_multi_and_unrolled_argument_errors(lib):
    # the many-right-hand-side and unrolled entry points reject bad arguments on the host,
    # before any CUDA call (the pointers below are never dereferenced)
    P = ctypes.c_void_p
    c = q._Codes(16, 16, 64, 128, 8, q.ld_words(64, 8))
    cy = q._Codes(16, 16, 64, 1, 8, q.ld_words(64, 8))
    prm = q._Params(2.0, 0.01, 32, 0)
    # the FP8 product and solve take codes of 2 or 4 bits only (8-bit centred codes are not exact in e4m3)
    assert lib.qiht_gemv_t_multi_fp8(ctypes.byref(c), P(256), 64, 4, P(256), 128, None, P(256), 1 << 30,
                                     None) == q.ERR_BITS
    fp8 = q._Params(2.0, 0.01, 32, q.SOLVE_FP8)
    assert lib.qiht_niht_solve_multi(ctypes.byref(c), ctypes.byref(c), (q._Codes * 1)(cy), 1, 4, 10,
                                     ctypes.byref(fp8), P(16), P(16), P(16), P(256), 1 << 30, None) == q.ERR_BITS
    assert lib.qiht_solve_multi_workspace_size(64, 128, 4, 3) > 0
    assert lib.qiht_solve_multi_workspace_size(16385, 128, 4, 3) == 0            # m above the limit
    assert lib.qiht_solve_multi_workspace_size(64, 128, 257, 3) == 0             # s above the limit
    assert lib.qiht_solve_multi_workspace_size(64, 128, 4, 0) == 0               # no right-hand side
    ys = (q._Codes * 2)(cy, cy)
    multi = lib.qiht_niht_solve_multi
    assert multi(ctypes.byref(c), ctypes.byref(c), ys, 2, 0, 10, ctypes.byref(prm), P(16), P(16), P(16),
                 P(256), 1 << 30, None) == q.ERR_ARG                              # s < 1
    assert multi(ctypes.byref(c), ctypes.byref(c), ys, 2, 4, 10, ctypes.byref(prm), None, P(16), P(16),
                 P(256), 1 << 30, None) == q.ERR_ARG                              # no X
    ybad = (q._Codes * 2)(cy, q._Codes(16, 16, 63, 1, 8, q.ld_words(63, 8)))
    assert multi(ctypes.byref(c), ctypes.byref(c), ybad, 2, 4, 10, ctypes.byref(prm), P(16), P(16), P(16),
                 P(256), 1 << 30, None) == q.ERR_ARG                              # an observation of 63 rows
    assert multi(ctypes.byref(c), ctypes.byref(c), ys, 2, 4, 10, ctypes.byref(prm), P(16), P(16), P(16),
                 None, 0, None) == q.ERR_WORKSPACE
    assert multi(ctypes.byref(c), ctypes.byref(c), ys, 2, 4, 10, ctypes.byref(prm), P(16), P(16), P(16),
                 P(272), 1 << 30, None) == q.ERR_WORKSPACE                        # not 256-byte aligned

    ws = lib.qiht_unrolled_workspace_size(2, 64, 128, 4, 5)
    assert ws > 0 and lib.qiht_unrolled_workspace_size(2, 64, 128, 4, 0) > 0     # K = 0 is valid
    assert lib.qiht_unrolled_workspace_size(0, 64, 128, 4, 5) == 0
    assert lib.qiht_unrolled_workspace_size(2, 16385, 128, 4, 5) == 0
    assert lib.qiht_unrolled_workspace_size(2, 64, 128, 65, 5) == 0              # s > m
    assert lib.qiht_unrolled_workspace_size(2, 64, 128, 4, -1) == 0
    Qa = (q._Codes * 2)(c, c)
    fwd, bwd = lib.qiht_unrolled_forward, lib.qiht_unrolled_backward
    assert fwd(Qa, Qa, 2, P(16), None, P(16), 4, 5, P(16), P(256), ws, None) == q.ERR_ARG       # no gain
    Qm = (q._Codes * 2)(c, q._Codes(16, 16, 64, 127, 8, q.ld_words(64, 8)))
    assert fwd(Qa, Qm, 2, P(16), P(16), P(16), 4, 5, P(16), P(256), ws, None) == q.ERR_ARG      # n differs
    Q4 = (q._Codes * 2)(c, q._Codes(16, 16, 64, 128, 4, q.ld_words(64, 4)))
    assert fwd(Q4, Q4, 2, P(16), P(16), P(16), 4, 5, P(16), P(256), ws, None) == q.ERR_ARG      # bits differ
    Q3 = (q._Codes * 2)(c, q._Codes(16, 16, 64, 128, 3, 4))
    assert fwd(Q3, Q3, 2, P(16), P(16), P(16), 4, 5, P(16), P(256), ws, None) == q.ERR_BITS
    assert fwd(Qa, Qa, 2, P(16), P(16), P(16), 4, 5, P(16), None, 0, None) == q.ERR_WORKSPACE
    assert fwd(Qa, Qa, 2, P(16), P(16), P(16), 4, 5, P(16), P(256), ws - 1, None) == q.ERR_WORKSPACE
    assert fwd(Qa, Qa, 2, P(16), P(16), P(16), 4, 5, P(16), P(272), ws, None) == q.ERR_WORKSPACE
    assert bwd(Qa, Qa, 2, P(16), P(16), P(16), 4, 5, None, P(16), P(16), P(16), P(256), ws,
               None) == q.ERR_ARG                                                # no Xbar


def test_fresh_argument_errors(lib):
    P = ctypes.c_void_p
    prm = q._Params(2.0, 0.01, 32, 0)
    ws = lib.qiht_solve_fresh_workspace_size(64, 128, 4, 8, 8)
    assert ws > 0
    assert lib.qiht_solve_fresh_workspace_size(16385, 128, 4, 8, 8) == 0         # m above the limit
    assert lib.qiht_solve_fresh_workspace_size(64, 128, 4, 3, 8) == 0            # bits
    assert lib.qiht_solve_fresh_workspace_size(64, 128, 65, 8, 8) == 0           # s > m
    fresh = lib.qiht_niht_solve_fresh
    args = dict(phi=P(16), ld=128, y=P(16), m=64, n=128, bp=8, by=8, seed=1, flags=0, s=4, iters=10)

    def call(**kw):
        a = {**args, **kw}
        return fresh(a["phi"], a["ld"], a["y"], a["m"], a["n"], a["bp"], a["by"], a["seed"], a["flags"], a["s"],
                     a["iters"], ctypes.byref(prm), P(16), P(16), P(16), None, kw.get("ws", P(256)),
                     kw.get("wsb", ws), None)
    assert call(bp=3) == q.ERR_BITS
    assert call(ld=100) == q.ERR_ARG                                           # row stride below n
    assert call(y=None) == q.ERR_ARG
    assert call(s=65) == q.ERR_ARG
    assert call(flags=64) == q.ERR_ARG                                         # unknown flag
    assert call(ws=None, wsb=0) == q.ERR_WORKSPACE
    assert call(wsb=ws - 1) == q.ERR_WORKSPACE


def test_fly_argument_errors(lib):
    # the on-the-fly operator's limits are checked on the host, before any CUDA call (the
    # pointers below are never dereferenced)
    P = ctypes.c_void_p
    ok = q._FlyOp(16, 16, 8, 16)                     # K = 8 baselines, 16 x 16 grid
    ldw = q.ld_words(16, 8)
    fq, fg = lib.qiht_fly_quantize, lib.qiht_gemv_t_fly
    assert fq(ctypes.byref(ok), 3, 0, 0, 0, 0, P(256), None, ldw, P(16), None) == q.ERR_BITS
    assert fg(ctypes.byref(ok), 5, 0, 0, 0, P(16), P(16), P(16), None) == q.ERR_BITS
    for bad in (q._FlyOp(16, 16, 6, 16),            # K not a multiple of 4
                q._FlyOp(16, 16, 0, 16),            # no baselines
                q._FlyOp(16, 16, 8200, 16),         # 2K above the row limit
                q._FlyOp(16, 16, 8, 24),            # g not a power of two
                q._FlyOp(16, 16, 8, 512),           # g above the limit
                q._FlyOp(None, 16, 8, 16), q._FlyOp(16, None, 8, 16)):
        assert fq(ctypes.byref(bad), 8, 0, 0, 0, 0, P(256), None, ldw, P(16), None) == q.ERR_ARG
        assert fg(ctypes.byref(bad), 8, 0, 0, 0, P(16), P(16), P(16), None) == q.ERR_ARG
    assert fq(ctypes.byref(ok), 8, 0, 0, 0, 0, P(256), None, ldw + 4, P(16), None) == q.ERR_ARG   # ld_words
    assert fq(ctypes.byref(ok), 8, 0, 0, 0, 0, P(260), None, ldw, P(16), None) == q.ERR_ARG       # unaligned
    assert fq(ctypes.byref(ok), 8, 0, 0, 1, 0, P(256), P(256), ldw, P(16), None) == q.ERR_ARG     # same buffer
    assert fq(ctypes.byref(ok), 8, 0, 0, 0, 64, P(256), None, ldw, P(16), None) == q.ERR_ARG      # unknown flag
    assert fg(ctypes.byref(ok), 8, 0, 0, 0, None, P(16), P(16), None) == q.ERR_ARG
    prm = q._Params(2.0, 0.01, 32, 0)
    sf = lib.qiht_niht_solve_fresh_fly
    big = q._FlyOp(16, 16, 8, 256)                  # n = 65536 columns: above the solve's limit
    assert sf(ctypes.byref(big), P(16), 8, 8, 1, 0, 4, 10, ctypes.byref(prm), P(16), P(16), P(16), None, P(256),
              1 << 30, None) == q.ERR_ARG
    assert sf(ctypes.byref(q._FlyOp(16, 16, 6, 16)), P(16), 8, 8, 1, 0, 4, 10, ctypes.byref(prm), P(16), P(16),
              P(16), None, P(256), 1 << 30, None) == q.ERR_ARG
    assert sf(ctypes.byref(ok), P(16), 3, 8, 1, 0, 4, 10, ctypes.byref(prm), P(16), P(16), P(16), None, P(256),
              1 << 30, None) == q.ERR_BITS


def test_sep_argument_errors(lib):
    # the separable operator's limits are checked on the host before any CUDA call
    P = ctypes.c_void_p
    prm = q._Params(2.0, 0.01, 32, 0)
    ws = lib.qiht_solve_separable_workspace_size(32, 300, 16)
    assert ws > 0
    assert lib.qiht_solve_separable_workspace_size(513, 300, 16) == 0            # N above the limit
    assert lib.qiht_solve_separable_workspace_size(32, 2000, 16) == 0            # M > N^2
    ok = q._SepOp(16, 16, 32, 300)
    sv = lib.qiht_niht_solve_separable

    def call(op=ok, bf=12, by=8, flags=0, s=16, iters=5, params=prm, wsb=ws, y=P(16)):
        return sv(ctypes.byref(op), y, bf, by, 1, flags, s, iters, ctypes.byref(params), P(16), P(16), P(16), None,
                  P(256), wsb, None)
    assert call(bf=1) == q.ERR_BITS and call(by=17) == q.ERR_BITS
    assert call(op=q._SepOp(16, 16, 513, 300)) == q.ERR_ARG
    assert call(op=q._SepOp(None, 16, 32, 300)) == q.ERR_ARG
    assert call(op=q._SepOp(16, 16, 32, 0)) == q.ERR_ARG
    assert call(s=601) == q.ERR_ARG                                              # s > m = 2M
    assert call(flags=64) == q.ERR_ARG
    assert call(y=None) == q.ERR_ARG
    assert call(params=q._Params(2.0, 0.01, 32, 0, 0.0, q.MU_CROSS, 0)) == q.ERR_ARG   # forward square only
    assert call(wsb=ws - 1) == q.ERR_WORKSPACE
    assert lib.qiht_sep_quantize_factor(ctypes.byref(ok), 20, 0, 0, 0, None, P(16), P(16), None) == q.ERR_BITS
    assert lib.qiht_sep_quantize_factor(ctypes.byref(ok), 12, 0, 0, 0, None, None, P(16), None) == q.ERR_ARG
    assert lib.qiht_sep_apply(ctypes.byref(ok), P(16), 0, P(16), P(16), P(256), 16, None) == q.ERR_WORKSPACE


def test_grid_levels_are_checked(lib):
    P = ctypes.c_void_p
    ld = q.ld_words(64, 8)
    prm = q._Params(2.0, 0.01, 32, 0)
    solve = lib.qiht_niht_solve
    for bits in (2, 4, 8):
        ldb = q.ld_words(64, bits)
        cy = q._Codes(16, 16, 64, 1, 8, ld)
        valid = {0, 2**bits, q.odd_levels(bits)}
        for levels in sorted(valid | {1, 2**bits - 1, q.odd_levels(bits) + 1, 2**bits + 1, -1}):
            ok = levels in valid
            c = q._Codes(16, 16, 64, 128, bits, ldb, levels, 0)
            # a valid grid gets as far as the workspace check; any other level count is an argument error
            want = q.ERR_WORKSPACE if ok else q.ERR_ARG
            assert solve(ctypes.byref(c), ctypes.byref(c), ctypes.byref(cy), 4, 10, ctypes.byref(prm), P(16),
                         P(16), P(16), None, None, 0, None) == want, (bits, levels)
            assert lib.qiht_gemv_t(ctypes.byref(c), P(16), P(16), None, 0, None) == want, (bits, levels)
    # the odd-grid flag is a known quantize flag (null input still fails the argument check)
    assert lib.qiht_quantize(None, 4, 4, 4, 8, 0, 0, q.ODD_LEVELS, P(16), 4, P(16), None) == q.ERR_ARG
    assert lib.qiht_quantize(P(16), 4, 4, 4, 8, 0, 0, 8, P(16), 4, P(16), None) == q.ERR_ARG


def test_struct_layout_matches_header(tmp_path):
    # the binding's ctypes structures have the sizes and field offsets the C compiler gives the header's
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "qiht.h"\n'
        'int main(void) { printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(qiht_codes), offsetof(qiht_codes, levels),'
        ' sizeof(qiht_problem), offsetof(qiht_problem, s), offsetof(qiht_problem, x), sizeof(qiht_report),'
        ' sizeof(qiht_params)); printf("%zu %zu %zu\\n", sizeof(qiht_fly_op), offsetof(qiht_fly_op, grid), sizeof(qiht_sep_op)); return 0; }\n')
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(q._Codes), q._Codes.levels.offset, ctypes.sizeof(q._Problem), q._Problem.s.offset,
            q._Problem.x.offset, ctypes.sizeof(q._Report), ctypes.sizeof(q._Params), ctypes.sizeof(q._FlyOp),
            q._FlyOp.grid.offset, ctypes.sizeof(q._SepOp)]
    assert got == want


def test_package_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(q, "_lib", None)
    monkeypatch.setattr(q, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        q.lib()
