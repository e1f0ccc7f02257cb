"""GPU parity of each streaming tile layout (amg_config.layout) on its own:
CSR row tiles, windowed CSR tiles, sliced-ELL tiles and the direct
sliced-ELL layout (no staging), each pinned by the
layout option and checked against the FP64 oracle through the V-cycle, the
solve, the adjoint and a numeric re-setup.  Matrices have at least 16384
rows (the streaming kernels' threshold) and ragged last tiles and slices."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M

pytestmark = pytest.mark.gpu

DEV = "cuda"
LAYOUTS = ["CSR", "WINDOWED", "SLICED_ELL", "ELL_DIRECT"]

CASES = {
    # n = 35937 = 32 * 1123 + 1: one row in the last slice
    "grf3d_33": lambda: M.diffusion3d_grf(N=33).A,
    # n = 32761: a last slice of 25 rows
    "poisson2d_181": lambda: M.poisson2d(181),
    # nonsymmetric (BiCGStab, hierarchy of A^T for the adjoint)
    "convdiff_29": lambda: M.convdiff3d_upwind(N=29).A,
    # level 1 (20,619 rows) streams too
    "grf3d_61": lambda: M.diffusion3d_grf(N=61).A,
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def solver(A, cfg):
    return api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values), cfg)


def check_layout(s, layout):
    """Every operator that streams runs the requested layout (level 0's A in
    particular, which fits all three at these sizes)."""
    ops = ["pre", "post", "P", "R"]
    for l in range(s.info().nlevels):
        for op in ops + (["krylov"] if l == 0 else []):
            p = s.plan(l, op)
            if p["rows_per_tile"] > 0 and (l == 0 and op in ("pre", "post", "krylov")):
                assert p["layout"] == layout, (l, op, p)
            if p["layout"] in ("SLICED_ELL", "ELL_DIRECT"):
                assert p["rows_per_tile"] % 32 == 0 and p["threads_per_row"] == 1


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_layout_parity(name, layout):
    A = CASES[name]()
    r = np.random.default_rng(1).uniform(-1, 1, A.n)
    zo = O.Hierarchy(A).vcycle(r)
    s = solver(A, {"layout": layout})
    check_layout(s, layout)
    z = s.vcycle(dev(r)).cpu().numpy()
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    sm = solver(A, {"layout": layout, "precision": "MIXED"})
    check_layout(sm, layout)
    zm = sm.vcycle(dev(r)).cpu().numpy()
    assert np.linalg.norm(zm - zo) <= 1e-5 * np.linalg.norm(zo)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("name", list(CASES))
def test_solve_and_adjoint_layout_parity(name, precision, layout):
    A = CASES[name]()
    ocfg = {"solver": 1} if name.startswith("convdiff") else {}
    cfg = {"solver": "BICGSTAB"} if name.startswith("convdiff") else {}
    cfg.update(layout=layout, precision=precision)
    rng = np.random.default_rng(7)
    b = rng.uniform(-1, 1, A.n)
    g = rng.uniform(-1, 1, A.n)
    _, io = O.Hierarchy(A, ocfg).solve(b)
    ht = O.Hierarchy(A, dict(ocfg, rtol=1e-13))
    xt, _ = ht.solve(b)
    lam_t, _, _ = ht.adjoint(xt, g, A.nnz)
    s = solver(A, cfg)
    x, info = s.solve(dev(b))
    assert info.status == 0 and info.rel_res_true <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    xn = x.cpu().numpy()
    assert np.linalg.norm(xn - xt) <= 1e-7 * np.linalg.norm(xt)
    lam, dA, ainfo = s.adjoint(x, dev(g))
    assert ainfo.status == 0 and ainfo.rel_res_true <= 1e-8
    lam = lam.cpu().numpy()
    assert np.linalg.norm(lam - lam_t) <= 1e-6 * np.linalg.norm(lam_t)
    rows = A.row_of()
    assert np.array_equal(dA.cpu().numpy(), -lam[rows] * xn[A.col_idx])


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_sliced_ell_resetup_lays_out_new_values(precision):
    """After a numeric re-setup the slot-order value copies follow the new
    values: the solve matches the oracle's re-set-up hierarchy."""
    A0 = M.diffusion3d_grf(N=33).A
    A1 = M.diffusion3d_grf(seed=9, N=33).A
    s = solver(A0, {"layout": "SLICED_ELL", "precision": precision})
    check_layout(s, "SLICED_ELL")
    b = np.random.default_rng(4).uniform(-1, 1, A1.n)
    s.resetup(dev(A1.values))
    x, info = s.solve(dev(b))
    _, io = O.Hierarchy(A0).resetup(A1.values).solve(b)
    xt, _ = O.Hierarchy(A1, {"rtol": 1e-13}).solve(b)
    assert info.status == 0 and info.rel_res_true <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    x = x.cpu().numpy()
    assert np.linalg.norm(x - xt) <= 1e-7 * np.linalg.norm(xt)


def test_sliced_ell_is_deterministic():
    """Each row's sum runs in a fixed slot order with no atomics: two
    sliced-ELL handles of one matrix give bitwise equal V-cycles."""
    A = M.diffusion3d_grf(N=33).A
    r = dev(np.random.default_rng(3).uniform(-1, 1, A.n))
    z1 = solver(A, {"layout": "SLICED_ELL"}).vcycle(r)
    z2 = solver(A, {"layout": "SLICED_ELL"}).vcycle(r)
    assert torch.equal(z1, z2)


def test_layout_option_is_validated():
    A = M.poisson2d(20)
    with pytest.raises(api.AMGError):
        solver(A, {"layout": 7})
