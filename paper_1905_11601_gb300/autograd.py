"""torch.autograd.Function over the Krylov map: y = A(U, Theta) x, differentiable in x and in the
base state (velocity U = (U, V, W) and temperature Theta).

The backward pass is hand-written: grad_x = A^T grad_y (kv_krylov_vector_adjoint) and
grad_(U, Theta) = d<grad_y, A x>/d(U, Theta) (kv_base_flow_gradient). Only x and the base state
are saved; the projections of grad_y are recomputed in the backward pass (checkpointing), so a
forward pass keeps no intermediate fields alive.
"""
from __future__ import annotations

import torch

from . import kv


class KrylovMap(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, theta, grid: "kv.Grid", velocity):
        base = torch.cat([velocity, theta.unsqueeze(0)]).contiguous()
        grid.set_base_flow(base)
        ctx.save_for_backward(x, theta, velocity)
        ctx.grid = grid
        return grid.krylov_vector(x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        x, theta, velocity = ctx.saved_tensors
        grid = ctx.grid
        grid.set_base_flow(torch.cat([velocity, theta.unsqueeze(0)]).contiguous())
        gy = gy.contiguous()
        gx = grid.krylov_vector_adjoint(gy) if ctx.needs_input_grad[0] else None
        gt = gu = None
        if ctx.needs_input_grad[1] or ctx.needs_input_grad[3]:
            gb, _ = grid.base_flow_gradient(x.contiguous(), gy, want_base=True, want_gr=False)
            gt = gb[3] if ctx.needs_input_grad[1] else None
            gu = gb[:3] if ctx.needs_input_grad[3] else None
        return gx, gt, None, gu


def krylov_map(x, theta, grid, velocity):
    """A(U, Theta) x through the CUDA path, differentiable in x, Theta and the base velocity."""
    return KrylovMap.apply(x, theta, grid, velocity)
