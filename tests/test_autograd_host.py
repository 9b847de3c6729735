"""Host logic of the unrolled autograd wrapper (paper_1802_04907_gb300.UnrolledQIHT), with a
stand-in for the CUDA operator: the backward uses the checkpoints of its own forward, recomputing
them when a later forward through the same operator replaced them."""
import torch

import paper_1802_04907_gb300 as q


class _FakeOp:
    """Records which inputs its checkpoints belong to; backward returns them tagged."""

    def __init__(self):
        self.generation = 0
        self.ckpt = None
        self.forwards = 0

    def forward(self, y, gre, gim):
        self.ckpt = y.clone()
        self.generation += 1
        self.forwards += 1
        return y[:, :2] * 1.0

    def backward(self, y, gre, gim, xbar):
        assert torch.equal(self.ckpt, y), "backward ran on another forward's checkpoints"
        return torch.ones_like(y) * self.ckpt.sum(), torch.zeros_like(gre), torch.zeros_like(gim)


def test_interleaved_forwards_recompute_the_checkpoints():
    op = _FakeOp()
    g = torch.ones(1, 3)
    y1 = torch.tensor([[1.0, 2.0, 3.0, 4.0, 5.0, 6.0]], requires_grad=True)
    y2 = torch.tensor([[10.0, 20.0, 30.0, 40.0, 50.0, 60.0]], requires_grad=True)
    x1 = q.UnrolledQIHT.apply(y1, g, g, op)
    x2 = q.UnrolledQIHT.apply(y2, g, g, op)
    (x1.sum() + x2.sum()).backward()
    assert op.forwards == 3                          # y1's checkpoints were recomputed once
    assert torch.all(y1.grad == 21.0) and torch.all(y2.grad == 210.0)


def test_single_forward_is_not_recomputed():
    op = _FakeOp()
    g = torch.ones(1, 3)
    y = torch.arange(6.0).reshape(1, 6).requires_grad_(True)
    q.UnrolledQIHT.apply(y, g, g, op).sum().backward()
    assert op.forwards == 1 and torch.all(y.grad == 15.0)
