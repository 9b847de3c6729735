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
    op = q.Unrolled(Q1s, Q1s, 4, 3)
    y, g = torch.zeros(2, 32), torch.zeros(2, 16)
    with pytest.raises(ValueError, match="y:"):
        op.forward(y, g, g)                                            # on the CPU
    with pytest.raises(ValueError, match="y:"):
        op.backward(y, g, g, torch.zeros(2, 32))
    assert op.generation == 0                                          # nothing ran


def test_fresh_solver_checks_its_inputs():
    with pytest.raises(ValueError, match="phi:"):
        q.niht_solve_fresh(torch.zeros(8, 16), torch.zeros(8), 8, 8, 1, 2, 3)
