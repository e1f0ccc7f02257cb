"""Error of every workload's GPU results against the FP64 oracle, at full size,
in both precision forms.

For each workload the GPU solves at rtol 1e-8 and runs the adjoint (Eq. 1-2)
with a seeded g; the oracle does the same at rtol 1e-8 and at rtol 1e-12 (the
reference solution).  Bars:
  * x: relative 2-norm error against the reference <= 1e-7; when a form
    misses it at rtol 1e-8 the solve is repeated at 1e-9 and 1e-10 and the
    rtol at which it passes is recorded (the bar must pass by 1e-10);
  * lambda = dL/db and dA = dL/dA: relative 2-norm error <= 1e-6;
  * entry by entry, max|e| / max|reference| no worse than twice the oracle's
    own at rtol 1e-8, with the 2-norm bar as a floor: a wrong value on a few
    rows (a ragged last tile, a slice boundary) fails here even when the
    norm hides it;
  * iterations within 2 of the oracle's at rtol 1e-8 (the mixed form too).
With AMG_ERROR_REPORT set, every (workload, form) appends one JSON record
with the measured errors to that file."""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M
from paper_2606_09001_b300 import _lib

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel2(a, ref):
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def relmax(a, ref):
    return float(np.abs(a - ref).max() / np.abs(ref).max())


def report(rec):
    path = os.environ.get("AMG_ERROR_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


WORKLOADS = {
    "C1_poisson2d_64": (lambda: M.poisson2d_64(), "PCG"),
    "C2_diffusion3d_grf_128": (lambda: M.diffusion3d_grf(), "PCG"),
    "C3_diffusion2d_logk_512": (lambda: M.diffusion2d_logk(), "PCG"),
    "C5_convdiff3d_upwind_160": (lambda: M.convdiff3d_upwind(), "BICGSTAB"),
    "tridiag_1e7": (lambda: M.tridiagonal_1e7(), "CG"),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_error_against_oracle(name):
    gen, solver = WORKLOADS[name]
    w = gen()
    A, b = w.A, w.b
    g = np.random.default_rng(7).uniform(-1, 1, A.n)
    osolver = _lib.SOLVERS[solver]
    h8 = O.Hierarchy(A, {"solver": osolver})
    x8, i8 = h8.solve(b)
    l8, d8, _ = h8.adjoint(x8, g, A.nnz)
    h8.close()
    h12 = O.Hierarchy(A, {"solver": osolver, "rtol": 1e-12})
    x12, _ = h12.solve(b)
    l12, d12, _ = h12.adjoint(x12, g, A.nnz)
    h12.close()
    own = {"x": relmax(x8, x12), "lambda": relmax(l8, l12), "dA": relmax(d8, d12)}
    own2 = {"x": rel2(x8, x12), "lambda": rel2(l8, l12), "dA": rel2(d8, d12)}
    rp, ci, v = dev(A.row_ptr), dev(A.col_idx), dev(A.values)
    bd, gd = dev(b), dev(g)
    forms = ("FP64",) if solver == "CG" else ("FP64", "MIXED")  # no V-cycle, no mixed form
    for form in forms:
        cfg = {"solver": solver, "precision": form}
        with api.Solver(rp, ci, v, cfg) as s:
            x, info = s.solve(bd)
            lam, dA, ainfo = s.adjoint(x, gd)
            x, lam, dA = x.cpu().numpy(), lam.cpu().numpy(), dA.cpu().numpy()
        assert info.status == 0 and info.rel_res_true <= 1e-8, (form, info)
        assert ainfo.status == 0 and ainfo.rel_res_true <= 1e-8, (form, ainfo)
        assert abs(info.iters - i8.iters) <= 2, (form, info.iters, i8.iters)
        err = {"x": rel2(x, x12), "lambda": rel2(lam, l12), "dA": rel2(dA, d12)}
        emax = {"x": relmax(x, x12), "lambda": relmax(lam, l12), "dA": relmax(dA, d12)}
        rtol_pass = 1e-8
        if err["x"] > 1e-7:
            rtol_pass = None
            for rt in (1e-9, 1e-10):
                with api.Solver(rp, ci, v, dict(cfg, rtol=rt)) as s2:
                    xr, _ = s2.solve(bd)
                if rel2(xr.cpu().numpy(), x12) <= 1e-7:
                    rtol_pass = rt
                    break
        report({"workload": name, "form": form, "solver": solver, "n": A.n, "iters": info.iters,
                "adjoint_iters": ainfo.iters, "oracle_iters": i8.iters, "rel_res_true": info.rel_res_true,
                "err_2norm": err, "err_max": emax, "oracle_own_2norm": own2, "oracle_own_max": own,
                "x_bar_1e-7_met_at_rtol": rtol_pass})
        assert rtol_pass is not None, (form, err)
        assert err["lambda"] <= 1e-6 and err["dA"] <= 1e-6, (form, err)
        floor = {"x": 1e-7, "lambda": 1e-6, "dA": 1e-6}
        for k in emax:
            assert emax[k] <= max(2.0 * own[k], floor[k]), (form, k, emax[k], own[k])


def test_error_batched_sampled():
    """The batched Poisson workload (256 systems x 8 right-hand sides) in both
    forms: sampled systems (the smallest, the largest and six between) with
    all 8 right-hand sides against the oracle run on each system alone."""
    w = M.batched_poisson2d()
    off = w.extra["sys_off"]
    sides = w.extra["sides"]
    order = np.argsort(sides, kind="stable")
    sample = sorted(set(int(order[q]) for q in np.linspace(0, len(order) - 1, 8).round().astype(int)))
    refs = {}
    for k in sample:
        Bk = M.poisson2d(int(sides[k]))
        r0, r1 = off[k], off[k + 1]
        h8, h12 = O.Hierarchy(Bk), O.Hierarchy(Bk, {"rtol": 1e-12})
        cols = []
        for r in range(8):
            bk = np.ascontiguousarray(w.b[r0:r1, r])
            x8, i8 = h8.solve(bk)
            x12, _ = h12.solve(bk)
            cols.append((x8, i8.iters, x12))
        refs[k] = cols
        h8.close()
        h12.close()
    for form in ("FP64", "MIXED"):
        s = api.BatchedSolver(dev(off), dev(w.A.row_ptr), dev(w.A.col_idx), dev(w.A.values), {"precision": form})
        X, its, rel, info = s.solve(dev(w.b))
        s.close()
        assert info.status == 0 and np.all(rel <= 1e-8), form
        X = X.cpu().numpy()
        worst2, worstm = 0.0, 0.0
        for k, cols in refs.items():
            r0, r1 = off[k], off[k + 1]
            for r, (x8, it8, x12) in enumerate(cols):
                xg = X[r0:r1, r]
                e2, em = rel2(xg, x12), relmax(xg, x12)
                worst2, worstm = max(worst2, e2), max(worstm, em)
                assert e2 <= 1e-7, (form, k, r, e2)
                assert em <= max(2.0 * relmax(x8, x12), 1e-7), (form, k, r, em)
                assert abs(int(its[k, r]) - it8) <= 2, (form, k, r, int(its[k, r]), it8)
        report({"workload": "C4_batched_poisson2d_256x8", "form": form, "systems_sampled": sample,
                "err_2norm": {"x": worst2}, "err_max": {"x": worstm}})
