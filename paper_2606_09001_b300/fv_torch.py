"""Differentiable assembly of the cell-centred finite-volume diffusion
operator in torch, so that a loss can be differentiated through the solve
with respect to per-cell log-conductivities (the inverse-problem workflow of
the paper's Sec. 3.2, on the 2D diffusion workload).

``fv_values(theta, A)`` returns the stored values of the CSR matrix built by
:func:`paper_2606_09001_b300.matrices.diffusion_fv` for ``k = exp(theta)``,
in the same storage order, as a differentiable function of ``theta``.  The
sparsity pattern is fixed, so the solver's setup cache key (the pattern) is
unchanged as theta moves.
"""
from __future__ import annotations

import torch


def _faces(k: torch.Tensor, axis: int):
    """Interior face coefficients 2 k_i k_j / (k_i + k_j) along ``axis``."""
    a = k.narrow(axis, 0, k.shape[axis] - 1)
    b = k.narrow(axis, 1, k.shape[axis] - 1)
    return 2.0 * a * b / (a + b)


def fv_values(theta: torch.Tensor) -> torch.Tensor:
    """CSR values (storage order of ``matrices.diffusion_fv``) of the 2D or 3D
    FV operator for k = exp(theta); theta has shape (N, N) or (N, N, N)
    indexed [y, x] / [z, y, x]."""
    k = torch.exp(theta)
    dim = k.dim()
    N = k.shape[0]
    n = k.numel()
    dev, dt = k.device, k.dtype
    # axis of the array for each grid direction d (x = 0 is the last axis)
    ax = {d: dim - 1 - d for d in range(dim)}
    zero = torch.zeros((), device=dev, dtype=dt)
    neg_cols, pos_cols = [], []
    diag = torch.zeros_like(k)
    # candidate order per row: -z, -y, -x, self, +x, +y, +z (ascending column)
    for d in reversed(range(dim)):  # negative neighbours
        a = ax[d]
        c = _faces(k, a)
        # face between cell and its -d neighbour, for cells with index >= 1 along a
        face = torch.cat([2.0 * k.narrow(a, 0, 1), c], dim=a)  # boundary face at index 0
        inside = torch.ones_like(k, dtype=torch.bool)
        inside.narrow(a, 0, 1).fill_(False)
        neg_cols.append((torch.where(inside, -face, zero), inside))
        diag = diag + face
    for d in range(dim):  # positive neighbours
        a = ax[d]
        c = _faces(k, a)
        face = torch.cat([c, 2.0 * k.narrow(a, N - 1, 1)], dim=a)  # boundary face at index N-1
        inside = torch.ones_like(k, dtype=torch.bool)
        inside.narrow(a, N - 1, 1).fill_(False)
        pos_cols.append((torch.where(inside, -face, zero), inside))
        diag = diag + face
    cols = neg_cols + [(diag, torch.ones_like(k, dtype=torch.bool))] + pos_cols
    vals = torch.stack([c[0].reshape(n) for c in cols], dim=1)
    mask = torch.stack([c[1].reshape(n) for c in cols], dim=1)
    return vals[mask]
