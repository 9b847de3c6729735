"""The allocation-free column-subset product, qiht_gemv_cols_static.

It serves callers that cannot allocate device memory when they need the product
(while a stream is being captured, inside real-time loops, in plug-ins whose host
owns all device memory): its scratch is a fixed array inside the library instead
of a workspace. Called through the C ABI, it must give the same z = Q[:, cols] c
as qiht_gemv_cols (within the FP32 bound used for that product's parity test),
on two calls in a row, since the array keeps the previous call's contents.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1802_04907_gb300 as q
import synth

pytestmark = pytest.mark.gpu


def _bound(A, cols, coef):
    mag = np.abs(A[:, cols]) @ np.abs(coef.astype(np.float64))
    return 1.1 * (2 * cols.size + 4) * 2.0**-24 * mag + 1e-30


def test_static_scratch_matches_workspace_version():
    lib = q.lib()
    m, n, bits = 4096, 3000, 4
    v = synth.random_floats((m, n), seed=21)
    Q = q.quantize(torch.from_numpy(v).cuda(), bits, 7, 1)
    codes, c = oracle.quantize(v, bits, 7, 1)
    A = oracle.dequantize(codes, bits, c)
    rng = np.random.Generator(np.random.PCG64(5))
    stream = torch.cuda.current_stream().cuda_stream
    cq = Q.c_struct()
    for count in (300, 77):                      # two calls in a row, different sizes
        cols = rng.choice(n, count, replace=False).astype(np.int32)
        coef = rng.standard_normal(count).astype(np.float32)
        cols_t = torch.from_numpy(cols).cuda()
        coef_t = torch.from_numpy(coef).cuda()
        z_ws = q.gemv_cols(Q, cols_t, coef_t)
        z = torch.full((m,), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.qiht_gemv_cols_static(ctypes.byref(cq), cols_t.data_ptr(), coef_t.data_ptr(), count,
                                       z.data_ptr(), stream)
        assert st == q.OK, q.status_string(st)
        torch.cuda.synchronize()
        got, ref = z.cpu().numpy().astype(np.float64), z_ws.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        bound = _bound(A, cols, coef)
        assert np.all(np.abs(got - ref) <= bound)
        exact = oracle.gemv_cols(A, cols, coef.astype(np.float64))
        assert np.all(np.abs(got - exact) <= bound)


def test_static_scratch_rejects_sizes_beyond_its_limit():
    lib = q.lib()
    m = 16384
    ld = q.ld_words(m, 8)
    c = q._Codes(256, 256, m, 8192, 8, ld)     # checked on the host: nothing is read or launched
    count = 4096
    assert lib.qiht_gemv_cols_workspace_size(m, count) > (2 << 20)
    st = lib.qiht_gemv_cols_static(ctypes.byref(c), ctypes.c_void_p(256), ctypes.c_void_p(256), count,
                                   ctypes.c_void_p(256), None)
    assert st == q.ERR_WORKSPACE
