"""GPU parity of classical Ruge-Stueben AMG (amg_config.amg_type = 1):
strength, PMIS C/F splitting and direct interpolation on the GPU against the
oracle's classical hierarchy -- the C/F map (as coarse indices), P, R and
every coarse operator bit for bit -- then solves and adjoints."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M
from paper_2606_09001_b300 import _lib

pytestmark = pytest.mark.gpu

DEV = "cuda"
CL = {"amg_type": "CLASSICAL"}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def solver(A, cfg):
    return api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values), cfg)


def ocfg(cfg):
    c = {"amg_type": 1}
    for k, v in cfg.items():
        if k == "solver":
            c[k] = _lib.SOLVERS[v]
        elif k not in ("precision", "layout", "amg_type", "fuse_coarse"):
            c[k] = v
    return c


CASES = {
    "poisson2d_37": lambda: M.poisson2d(37),
    "grf3d_24": lambda: M.diffusion3d_grf(N=24).A,
    "logk2d_48": lambda: M.diffusion2d_logk(N=48).A,
    "convdiff_14": lambda: M.convdiff3d_upwind(N=14).A,
    # streaming kernels on level 0
    "grf3d_33": lambda: M.diffusion3d_grf(N=33).A,
    "poisson2d_181": lambda: M.poisson2d(181),
}


def solver_cfg(name):
    return {"solver": "BICGSTAB"} if name.startswith("convdiff") else {}


@pytest.mark.parametrize("name", list(CASES))
def test_classical_hierarchy_bit_exact(name):
    A = CASES[name]()
    cfg = dict(CL, **solver_cfg(name))
    h = O.Hierarchy(A, ocfg(cfg))
    s = solver(A, cfg)
    assert s.info().nlevels == h.nlevels >= 3
    for l in range(h.nlevels):
        lv = h.level(l)
        rp, ci, v, _ = s.level(l, "A")
        assert np.array_equal(rp, lv.A.row_ptr) and np.array_equal(ci, lv.A.col_idx), f"A{l} pattern"
        assert np.array_equal(v.view(np.int64), lv.A.values.view(np.int64)), f"A{l} values"
        if l < h.nlevels - 1:
            assert np.array_equal(s.aggregates(l), lv.agg), f"C/F map {l}"
            for which, ref in (("P", lv.P), ("R", lv.R)):
                rp, ci, v, _ = s.level(l, which)
                assert np.array_equal(rp, ref.row_ptr) and np.array_equal(ci, ref.col_idx), f"{which}{l} pattern"
                assert np.array_equal(v.view(np.int64), ref.values.view(np.int64)), f"{which}{l} values"


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("name", list(CASES))
def test_classical_solve_parity(name, precision):
    A = CASES[name]()
    cfg = dict(CL, precision=precision, **solver_cfg(name))
    b = np.random.default_rng(5).uniform(-1, 1, A.n)
    _, io = O.Hierarchy(A, ocfg(cfg)).solve(b)
    xt, _ = O.Hierarchy(A, dict(ocfg(cfg), rtol=1e-13)).solve(b)
    x, info = solver(A, cfg).solve(dev(b))
    assert info.status == 0 and io.status == 0 and info.rel_res_true <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    assert np.linalg.norm(x.cpu().numpy() - xt) <= 1e-7 * np.linalg.norm(xt)


@pytest.mark.parametrize("name", ["convdiff_14", "grf3d_24"])
def test_classical_adjoint_parity(name):
    A = CASES[name]()
    cfg = dict(CL, **solver_cfg(name))
    rng = np.random.default_rng(3)
    b, g = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    ht = O.Hierarchy(A, dict(ocfg(cfg), rtol=1e-13))
    xt, _ = ht.solve(b)
    lam_t, _, _ = ht.adjoint(xt, g, A.nnz)
    s = solver(A, cfg)
    x, _ = s.solve(dev(b))
    lam, dA, info = s.adjoint(x, dev(g))
    assert info.status == 0 and info.rel_res_true <= 1e-8
    lam = lam.cpu().numpy()
    assert np.linalg.norm(lam - lam_t) <= 1e-6 * np.linalg.norm(lam_t)
    assert np.array_equal(dA.cpu().numpy(), -lam[A.row_of()] * x.cpu().numpy()[A.col_idx])


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("pair", ["grf3d_24", "grf3d_33", "convdiff_14"])
def test_classical_resetup_bit_exact(pair, precision):
    """Classical re-setup: the C/F map and P's pattern kept, weights and every
    coarse operator recomputed, bit for bit against the oracle's re-setup."""
    if pair.startswith("grf3d"):
        N = int(pair.split("_")[1])
        A0, A1 = M.diffusion3d_grf(N=N).A, M.diffusion3d_grf(seed=9, N=N).A
        cfg = dict(CL, precision=precision)
    else:
        A0 = CASES[pair]()
        rng = np.random.default_rng(13)
        A1 = M.CSR(A0.row_ptr, A0.col_idx, A0.values * rng.uniform(0.8, 1.25, A0.nnz))
        cfg = dict(CL, precision=precision, solver="BICGSTAB")
    s = solver(A0, cfg)
    s.resetup(dev(A1.values))
    h = O.Hierarchy(A0, ocfg(cfg)).resetup(A1.values)
    assert s.info().nlevels == h.nlevels
    for l in range(h.nlevels):
        lv = h.level(l)
        rp, ci, v, _ = s.level(l, "A")
        assert np.array_equal(ci, lv.A.col_idx) and np.array_equal(v.view(np.int64), lv.A.values.view(np.int64)), l
        if l < h.nlevels - 1:
            assert np.array_equal(s.aggregates(l), lv.agg)
            for which, ref in (("P", lv.P), ("R", lv.R)):
                rp, ci, v, _ = s.level(l, which)
                assert np.array_equal(ci, ref.col_idx)
                assert np.array_equal(v.view(np.int64), ref.values.view(np.int64)), (which, l)
    b = np.random.default_rng(4).uniform(-1, 1, A1.n)
    x, info = s.solve(dev(b))
    _, io = h.solve(b)
    assert info.status == 0 and info.rel_res_true <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)


def test_classical_limits():
    A = M.poisson2d(40)
    blocks = [M.poisson2d(10), M.poisson2d(12)]
    Ab, off = M.block_diag(blocks)
    with pytest.raises(api.AMGError) as e:
        api.BatchedSolver(dev(off), dev(Ab.row_ptr), dev(Ab.col_idx), dev(Ab.values), CL)
    assert e.value.code == _lib.AMG_ERR_UNSUPPORTED
    with pytest.raises(api.AMGError):
        solver(A, {"amg_type": 5})
