"""Differentiable x = A(theta)^{-1} b for A(theta) = sum_e theta_e R_e^T K_e R_e.

The backward pass reuses the forward hierarchy for the adjoint solve A lambda = dL/dx and
forms dL/dtheta_e = -lambda_e^T K_e x_e in the library's element kernel (this follows from
dx/dtheta_e = -A^{-1} R_e^T K_e R_e x and the symmetry of A); dL/db = lambda.
"""
from __future__ import annotations

import torch

from .lsamg import Lsamg


class LsamgSolve(torch.autograd.Function):
    """apply(theta, b, n, elem_dofs, K, opts_dict) -> x  (all CUDA float64 tensors)."""

    @staticmethod
    def forward(ctx, theta, b, n, elem_dofs, K, opts):
        opts = dict(opts or {})
        mode = opts.pop("mode", -1)
        amg = Lsamg(n, elem_dofs, K, coef=theta.detach(), **opts)
        x, its, rel, rc = amg.solve(b.detach(), mode=mode, raise_on_noconv=True)
        ctx.amg = amg
        ctx.mode = mode
        ctx.save_for_backward(x)
        ctx.info = dict(forward_iters=its, forward_relres=rel)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        amg = ctx.amg
        lam, its, rel, rc = amg.solve(gx.contiguous(), mode=ctx.mode, raise_on_noconv=True)
        g = amg.elem_grad(lam, x)
        amg.close()
        ctx.amg = None
        return g, lam, None, None, None, None


def solve_with_grad(theta, b, n, elem_dofs, K, **opts):
    return LsamgSolve.apply(theta, b, n, elem_dofs, K, opts)
