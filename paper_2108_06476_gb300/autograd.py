"""torch.autograd wrapper of the rhs: forward dg_rhs, backward dg_rhs_vjp.

    du = RhsFn.apply(mesh, u)      # u: float64 CUDA tensor, requires_grad
    loss = (du * w).sum(); loss.backward()   # u.grad = (d rhs/d u)^T w

Both directions run the library's CUDA kernels; the backward pass recomputes
the two-point flux Jacobians instead of storing anything from the forward.
"""
from __future__ import annotations

import torch


class RhsFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mesh, u):
        ctx.mesh = mesh
        ctx.save_for_backward(u)
        return mesh.rhs(u.detach().contiguous()).to(torch.float64)

    @staticmethod
    def backward(ctx, w):
        (u,) = ctx.saved_tensors
        ubar = ctx.mesh.rhs_vjp(u.detach().contiguous(), w.to(torch.float64).contiguous())
        return None, ubar


def rhs(mesh, u):
    return RhsFn.apply(mesh, u)
