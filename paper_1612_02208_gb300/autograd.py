"""Differentiable Stokes-IB solve: torch.autograd.Function over the C ABI.

forward(g, kappa, X) -> w solves L_IB(X, kappa) w = b(g, X, kappa) (Eq. matrix-impib) with the
library's FGMRES + multigrid; backward(dl/dw) solves the adjoint system L_IB^T lam = dl/dw with
sib_solve_transpose (L_IB is symmetric, so this is the forward solve's FGMRES and V-cycle) and
evaluates dl/dkappa and dl/dX with sib_grad, which recomputes the spreading weights from X instead
of storing them.  dl/dg = lam.

All tensors live on the solver's CUDA device in float64; this module only marshals arguments.
"""
from __future__ import annotations

import torch

from . import sib


class StokesIBSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, kappa, X, solver, edges):
        token = object()
        _configure(solver, X, edges, kappa, token)
        w = solver.solve(g.detach().contiguous())
        ctx.solver = solver
        ctx.edges = edges
        ctx.token = token
        ctx.save_for_backward(w, kappa.detach(), X.detach())
        return w

    @staticmethod
    def backward(ctx, grad_w):
        w, kappa, X = ctx.saved_tensors
        solver = ctx.solver
        if getattr(solver, "_ad_token", None) is not ctx.token:   # another forward reconfigured it
            _configure(solver, X, ctx.edges, kappa, ctx.token)
        lam = solver.solve_transpose(grad_w.detach().contiguous())
        dkappa, dX = solver.grad(w, lam)
        return lam, dkappa, dX, None, None


def _configure(solver, X, edges, kappa, token):
    """Point the solver at (X, kappa) and run its set-up; remember which forward did it."""
    solver.set_structure(X.detach().contiguous(), edges, kappa.detach().contiguous())
    solver.setup()
    solver._ad_token = token


def stokes_ib_solve(solver: "sib.Solver", g: torch.Tensor, kappa: torch.Tensor, X: torch.Tensor,
                    edges: torch.Tensor) -> torch.Tensor:
    """w = L_IB(X, kappa)^{-1} b(g, X, kappa), differentiable in g, kappa and X."""
    return StokesIBSolve.apply(g, kappa, X, solver, edges)
