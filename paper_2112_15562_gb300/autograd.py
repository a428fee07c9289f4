"""Differentiable forms of the sensitivity products and the Gramian.

``G(op, m)`` is ``d = A m`` (gj_g_forward) with the hand-written adjoint product
(gj_g_adjoint) as its backward; ``GT(op, r)`` is the reverse pairing; ``gramian``
returns the FP64 value of Eq. (Gramian) and back-propagates through its ascent
directions (RRCG:2-3 give half the gradient).  Only argument marshalling happens
here: every product runs in the CUDA library.
"""
from __future__ import annotations

import torch

from .api import g_adjoint, g_forward, gramian_value_grad


class _GForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, op):
        ctx.op = op
        return g_forward(op, m.contiguous())

    @staticmethod
    def backward(ctx, grad_d):
        grad_m = g_adjoint(ctx.op, grad_d.contiguous()) if ctx.needs_input_grad[0] else None
        return grad_m, None


class _GAdjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r, op):
        ctx.op = op
        return g_adjoint(op, r.contiguous())

    @staticmethod
    def backward(ctx, grad_g):
        grad_r = g_forward(ctx.op, grad_g.contiguous()) if ctx.needs_input_grad[0] else None
        return grad_r, None


class _Gramian(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m1, m2):
        S, l1, l2 = gramian_value_grad(m1.contiguous(), m2.contiguous(), want_dirs=True)
        ctx.save_for_backward(l1, l2)
        return S.reshape(())

    @staticmethod
    def backward(ctx, grad_S):
        l1, l2 = ctx.saved_tensors
        g = 2.0 * grad_S
        return (g * l1).to(l1.dtype), (g * l2).to(l2.dtype)


def G(op, m: torch.Tensor) -> torch.Tensor:
    """d = A m, differentiable in m (backward: A^T)."""
    return _GForward.apply(m, op)


def GT(op, r: torch.Tensor) -> torch.Tensor:
    """g = A^T r, differentiable in r (backward: A)."""
    return _GAdjoint.apply(r, op)


def gramian(m1: torch.Tensor, m2: torch.Tensor) -> torch.Tensor:
    """S_G(m1, m2) as an FP64 scalar tensor, differentiable in both models."""
    return _Gramian.apply(m1, m2)
