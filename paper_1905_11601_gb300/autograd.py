"""torch.autograd.Function over the Krylov map: y = A(Theta) x, differentiable in x and in the
base-flow temperature Theta (the base velocity is held fixed by the grid).

The backward pass is hand-written: grad_x = A^T grad_y (kv_krylov_vector_adjoint) and
grad_Theta = d<grad_y, A x>/d Theta (kv_base_flow_gradient). Only x and Theta are saved; the
projections of grad_y are recomputed in the backward pass (checkpointing), so a forward pass
keeps no intermediate fields alive.
"""
from __future__ import annotations

import torch

from . import kv


class KrylovMap(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, theta, grid: "kv.Grid", velocity):
        base = torch.cat([velocity, theta.unsqueeze(0)]).contiguous()
        grid.set_base_flow(base)
        ctx.save_for_backward(x, theta)
        ctx.grid, ctx.velocity = grid, velocity
        return grid.krylov_vector(x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        x, theta = ctx.saved_tensors
        grid = ctx.grid
        grid.set_base_flow(torch.cat([ctx.velocity, theta.unsqueeze(0)]).contiguous())
        gy = gy.contiguous()
        gx = grid.krylov_vector_adjoint(gy) if ctx.needs_input_grad[0] else None
        gt = None
        if ctx.needs_input_grad[1]:
            gt, _ = grid.base_flow_gradient(x.contiguous(), gy, want_theta=True, want_gr=False)
        return gx, gt, None, None


def krylov_map(x, theta, grid, velocity):
    """A(Theta) x through the CUDA path, differentiable in x and Theta."""
    return KrylovMap.apply(x, theta, grid, velocity)
