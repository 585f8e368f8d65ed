"""The autograd Functions of grape.py, on the CPU with a stand-in table.

The Functions only chain libredo's gradient to an upstream gradient; their arithmetic is the
chain rule.  A stand-in table with a smooth fidelity whose gradient it knows exactly
(quantizer passed through, F_b = sum sin(a u_bnk), dF_b/du_bnk = a cos(a u_bnk)) lets
``torch.autograd.gradcheck`` check every vector-Jacobian product, with random upstream
gradients, against finite differences.
"""
import torch
from torch.autograd import gradcheck

from paper_1707_02162_gb300.grape import RedoFidelity, RedoPhaseFidelity, RedoStateFidelity


class _SmoothTable:
    a, b = 0.7, 1.3

    def quantize(self, u):
        return u.clone()

    def fidelity_grad(self, q, target, prec, checkpoint_every=0):
        return torch.sin(self.a * q).sum(dim=(1, 2)), self.a * torch.cos(self.a * q)

    def state_grad(self, q, psi0, psi_target, prec):
        return self.fidelity_grad(q, None, prec)

    def fidelity_grad_phase(self, q, phi, target, prec, checkpoint_every=0):
        F = torch.sin(self.a * q).sum(dim=(1, 2)) + torch.cos(self.b * phi * q).sum(dim=(1, 2))
        gA = self.a * torch.cos(self.a * q) - self.b * phi * torch.sin(self.b * phi * q)
        gP = -self.b * q * torch.sin(self.b * phi * q)
        return F, gA, gP


def _u(seed, shape=(3, 4, 2)):
    g = torch.Generator().manual_seed(seed)
    return torch.rand(shape, generator=g, dtype=torch.float64).mul_(2).sub_(1).requires_grad_(True)


def test_unitary_fidelity_function_chain_rule():
    t = _SmoothTable()
    assert gradcheck(lambda u: RedoFidelity.apply(u, t, None, "fp64", 0), (_u(0),), eps=1e-6, atol=1e-8)


def test_state_fidelity_function_chain_rule():
    t = _SmoothTable()
    assert gradcheck(lambda u: RedoStateFidelity.apply(u, t, None, None, "fp64"), (_u(1),), eps=1e-6, atol=1e-8)


def test_phase_fidelity_function_chain_rule_in_both_inputs():
    t = _SmoothTable()
    assert gradcheck(lambda A, P: RedoPhaseFidelity.apply(A, P, t, None, "fp64", 0), (_u(2), _u(3)),
                     eps=1e-6, atol=1e-8)


def test_upstream_weights_scale_each_pulse():
    t = _SmoothTable()
    u = _u(4)
    w = torch.tensor([0.5, -2.0, 0.0], dtype=torch.float64)
    (RedoFidelity.apply(u, t, None, "fp64", 0) * w).sum().backward()
    assert torch.allclose(u.grad, w[:, None, None] * t.a * torch.cos(t.a * u.detach()), rtol=0, atol=0)
