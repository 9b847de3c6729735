"""The Python wrappers refuse tensors of the wrong size, type, device or layout before any
launch (the kernels take raw pointers and would read out of bounds). Checked on the CPU:
every call below raises before the library is asked to launch anything."""
import pytest
import torch

import paper_1802_04907_gb300 as q


def _codes(rows, cols, bits=8):
    words = torch.zeros(cols * q.ld_words(rows, bits), dtype=torch.int32)
    return q.Codes(words, torch.ones(1), rows, cols, bits)


def test_vector_products_check_their_operands():
    Q = _codes(64, 40)
    with pytest.raises(ValueError, match="r:"):
        q.gemv_t(Q, torch.zeros(64))                                   # on the CPU
    with pytest.raises(ValueError, match="r:"):
        q.gemv_t(Q, torch.zeros(63))                                   # wrong length
    with pytest.raises(ValueError, match="r:"):
        q.gemv_t(Q, torch.zeros(64, dtype=torch.float64))              # wrong type
    with pytest.raises(ValueError, match="cols:"):
        q.gemv_cols(Q, torch.zeros(3, dtype=torch.int64), torch.zeros(3))
    with pytest.raises(ValueError, match="a:"):
        q.top_s(torch.zeros(10), 3)
    with pytest.raises(ValueError, match="r:"):
        q.gemv_t_prescaled(Q, torch.zeros(64), torch.zeros(1), torch.zeros(40))


def test_matrix_product_checks_its_operands():
    Q = _codes(64, 40)
    with pytest.raises(ValueError, match="R:"):
        q.gemv_t_multi(Q, torch.zeros(5, 64))                          # on the CPU
    with pytest.raises(ValueError, match="R:"):
        q.gemv_t_multi(Q, torch.zeros(5, 65))                          # rows do not match
    with pytest.raises(ValueError, match="R:"):
        q.gemv_t_multi(Q, torch.zeros(64, 5).t())                      # column stride 5


def test_unrolled_checks_its_operands():
    Q1s = [_codes(16, 32), _codes(16, 32)]
    with pytest.raises(ValueError, match="Codes.words"):
        q.Unrolled(Q1s, Q1s, 4, 3)                                     # codes on the CPU
    op = object.__new__(q.Unrolled)                                    # the operand checks alone
    op.P, op.m, op.n, op.generation = 2, 16, 32, 0
    y, g = torch.zeros(2, 32), torch.zeros(2, 16)
    with pytest.raises(ValueError, match="y:"):
        op.forward(y, g, g)                                            # on the CPU
    with pytest.raises(ValueError, match="y:"):
        op.backward(y, g, g, torch.zeros(2, 32))
    assert op.generation == 0                                          # nothing ran


def test_codes_descriptor_checks_its_buffers():
    # the kernels read cols * ld_words words and one scale through raw pointers
    good = _codes(64, 40)
    for bad in (q.Codes(good.words[:-4], good.scale, 64, 40, 8),                 # too short (a slice)
                q.Codes(good.words.to(torch.int64), good.scale, 64, 40, 8),      # wrong type
                q.Codes(good.words, good.scale, 64, 40, 8),                      # on the CPU
                q.Codes(good.words, good.scale, 64, 40, 3)):                     # bits
        with pytest.raises(ValueError, match="Codes"):
            bad.c_struct()


class _FakeStream:
    def __init__(self, handle):
        self.cuda_stream = handle
        self.waited_for = []

    def wait_stream(self, other):
        self.waited_for.append(other.cuda_stream)


def test_explicit_stream_waits_for_the_current_stream():
    # buffers a wrapper takes from the caching allocator come from the current stream's pool:
    # work launched on another stream must first wait for the current stream's queued work
    cur, other = _FakeStream(11), _FakeStream(22)
    assert q._stream(other, current=cur) == 22
    assert other.waited_for == [11]
    assert q._stream(cur, current=cur) == 11                          # the current stream: no wait
    assert cur.waited_for == []
    assert q._stream(None, current=cur) == 11


def test_fresh_buffers_are_recorded_on_a_foreign_stream():
    recorded = []

    class _T:
        device = "cuda:0"

        def record_stream(self, s):
            recorded.append(s.cuda_stream)

    cur, other = _FakeStream(11), _FakeStream(22)
    q._hold(_T(), other, current=cur)
    q._hold(_T(), cur, current=cur)
    q._hold(_T(), None, current=cur)
    assert recorded == [22]


def test_fresh_solver_checks_its_inputs():
    with pytest.raises(ValueError, match="phi:"):
        q.niht_solve_fresh(torch.zeros(8, 16), torch.zeros(8), 8, 8, 1, 2, 3)
