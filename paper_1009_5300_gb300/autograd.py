"""torch.autograd.Function for the conductance G(V) at one energy.

The forward pass sets the local potential, then runs the library's
iobm_grad_V, which solves the forward waves and the adjoint waves
A lambda_o = w_o (A = A^T) in one batch and accumulates dG/dV(r) in FP64 on
the device; backward scales that gradient by the incoming grad_output.
"""
from __future__ import annotations

import torch

from .solver import IOBMSolver


class IOBMConductance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V: torch.Tensor, solver: IOBMSolver, E: float):
        solver.set_potential(V)
        if V.requires_grad:
            g, G = solver.grad_V(E)
            ctx.save_for_backward(g)
        else:
            res = solver.solve([E])
            G = float(res.G[0])
            ctx.save_for_backward(None)
        return torch.tensor(G, dtype=torch.float64, device=V.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        if g is None:
            return None, None, None
        return (grad_out * g).to(dtype=torch.float64), None, None


def conductance(V: torch.Tensor, solver: IOBMSolver, E: float) -> torch.Tensor:
    """G(V) in G_0 at energy E, differentiable with respect to V ([nz][ny][nx])."""
    return IOBMConductance.apply(V, solver, E)
