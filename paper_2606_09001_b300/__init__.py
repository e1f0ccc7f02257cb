"""B300-native smoothed-aggregation AMG-preconditioned Krylov solver with a
reverse-mode adjoint (the method of the JAX-AMG paper, rebuilt on hand-written
sm_103a CUDA kernels behind a C ABI, include/amg_b300.h).

    from paper_2606_09001_b300 import Solver, solve, amg_solve
"""
from __future__ import annotations

__all__ = ["Solver", "BatchedSolver", "solve", "amg_solve", "SetupCache", "Info", "AMGError", "make_config"]


def __getattr__(name):
    # The CUDA-facing modules import torch; load them on first use so that
    # the input generators (matrices) import without it.
    if name in ("Solver", "BatchedSolver", "solve", "SetupCache", "Info", "AMGError", "make_config"):
        from . import api
        return getattr(api, name)
    if name == "amg_solve":
        from .autograd import amg_solve
        return amg_solve
    raise AttributeError(name)
