"""Differentiable solve: a torch.autograd.Function whose backward is the
paper's adjoint (Sec. 2.1 "JAX integration", Eq. 1-2), computed by the CUDA
library: A^T lambda = dL/dx, dL/db = lambda, dL/dA = -lambda x^T restricted
to the stored pattern.  The hierarchy is taken from the setup cache, so a
symmetric A reuses its forward hierarchy in the backward pass and a
nonsymmetric A builds (once) a hierarchy of A^T.  New values on the same
pattern re-set the cached hierarchy up (Sec. 2.1); a backward pass whose
handle was re-set up or evicted since its forward pass restores it for the
forward's values first."""
from __future__ import annotations

import torch

from .api import SetupCache, default_cache, make_config


class AMGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, b, row_ptr, col_idx, cfg, cache):
        solver = cache.get(row_ptr, col_idx, values.detach(), cfg)
        x, info = solver.solve(b.detach().contiguous())
        ctx.solver, ctx.generation = solver, solver.generation
        ctx.inputs = (row_ptr, col_idx, values.detach(), cfg, cache)
        ctx.info = info
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        need_A, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        solver = ctx.solver
        if getattr(solver, "_h", None) is None or solver.generation != ctx.generation:
            row_ptr, col_idx, values, cfg, cache = ctx.inputs
            solver = cache.get(row_ptr, col_idx, values, cfg)
        lam, dA, _ = solver.adjoint(x, gx.contiguous(), want_lambda=True, want_dA=need_A)
        return (dA if need_A else None), (lam if need_b else None), None, None, None, None


def amg_solve(row_ptr: torch.Tensor, col_idx: torch.Tensor, values: torch.Tensor, b: torch.Tensor,
              config: dict | None = None, cache: SetupCache = default_cache) -> torch.Tensor:
    """x = A^-1 b, differentiable with respect to ``values`` (the stored
    entries of A, in CSR order) and ``b``."""
    return AMGSolve.apply(values, b, row_ptr, col_idx, make_config(config), cache)
