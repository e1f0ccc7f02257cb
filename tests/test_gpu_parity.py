"""GPU parity: the CUDA library (called through the C ABI) against the FP64
CPU oracle on the same seeded inputs.

Bar: integer outputs (aggregates, sparsity patterns) bit-exact; hierarchy
values bit-exact too (both sides add in the same order with separately
rounded operations); solution, V-cycle and adjoint within the tolerances
stated at each test."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M
from paper_2606_09001_b300 import _lib

pytestmark = pytest.mark.gpu

DEV = "cuda"


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def gpu_solver(A, cfg=None):
    return api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values), cfg)


def ocfg(cfg):
    """The oracle's configuration for a library configuration dict."""
    c = dict(cfg or {})
    c.pop("precision", None)
    c.pop("layout", None)
    c.pop("fuse_coarse", None)
    if isinstance(c.get("solver"), str):
        c["solver"] = _lib.SOLVERS[c["solver"]]
    if isinstance(c.get("smoother"), str):
        c["smoother"] = _lib.SMOOTHERS[c["smoother"]]
    return c


SMALL_CASES = {
    "poisson2d_64": lambda: M.poisson2d_64().A,
    "poisson2d_37": lambda: M.poisson2d(37),
    "poisson3d_17": lambda: M.poisson3d(17),
    "grf3d_24": lambda: M.diffusion3d_grf(N=24).A,
    "logk2d_48": lambda: M.diffusion2d_logk(N=48).A,
    "convdiff_14": lambda: M.convdiff3d_upwind(N=14).A,
    "tridiag_1000": lambda: M.tridiagonal_matrix(1000, 2.5),
}

# Large enough (>= 16384 rows) for the bulk-copy streaming kernels, with a
# ragged last tile; grf3d_61 also streams on level 1 (20,619 rows).
STREAM_CASES = {
    "grf3d_33": lambda: M.diffusion3d_grf(N=33).A,
    "poisson2d_181": lambda: M.poisson2d(181),
    "convdiff_29": lambda: M.convdiff3d_upwind(N=29).A,
    "grf3d_61": lambda: M.diffusion3d_grf(N=61).A,
}
SMALL_CASES.update(STREAM_CASES)


def compare_hierarchy(A, cfg=None):
    h = O.Hierarchy(A, ocfg(cfg))
    s = gpu_solver(A, cfg)
    info = s.info()
    assert info.nlevels == h.nlevels
    for l in range(h.nlevels):
        lv = h.level(l)
        rp, ci, v, shape = s.level(l, "A")
        assert np.array_equal(rp, lv.A.row_ptr), f"A{l} row_ptr"
        assert np.array_equal(ci, lv.A.col_idx), f"A{l} col_idx"
        assert np.array_equal(v.view(np.int64), lv.A.values.view(np.int64)), f"A{l} values (bitwise)"
        if l < h.nlevels - 1:
            assert np.array_equal(s.aggregates(l), lv.agg), f"aggregates level {l}"
            for which, ref in (("P", lv.P), ("R", lv.R)):
                rp, ci, v, _ = s.level(l, which)
                assert np.array_equal(rp, ref.row_ptr) and np.array_equal(ci, ref.col_idx), f"{which}{l} pattern"
                assert np.array_equal(v.view(np.int64), ref.values.view(np.int64)), f"{which}{l} values"
    return h, s


@pytest.mark.parametrize("name", list(SMALL_CASES))
def test_hierarchy_bit_exact(name):
    A = SMALL_CASES[name]()
    cfg = {"solver": "BICGSTAB"} if name.startswith("convdiff") else None
    compare_hierarchy(A, cfg)


def test_hierarchy_bit_exact_l1_and_small_coarse():
    compare_hierarchy(M.poisson3d(12), {"smoother": "L1_JACOBI", "coarse_max": 8})


@pytest.mark.parametrize("name,cfg", [
    ("poisson2d_64", {}),
    ("poisson2d_37", {}),
    ("grf3d_24", {}),
    ("logk2d_48", {}),
    ("convdiff_14", {"solver": "BICGSTAB"}),
    ("tridiag_1000", {"solver": "CG"}),
    ("convdiff_14", {"solver": "BICGSTAB_NOPREC", "max_iter": 2000}),
    ("grf3d_33", {}),
    ("poisson2d_181", {}),
    ("convdiff_29", {"solver": "BICGSTAB"}),
    ("grf3d_61", {}),
    ("poisson2d_181", {"solver": "CG", "max_iter": 5000}),
])
def test_solve_parity(name, cfg):
    A = SMALL_CASES[name]()
    b = np.random.default_rng(5).uniform(-1, 1, A.n)
    h = O.Hierarchy(A, ocfg(cfg))
    xo, io = h.solve(b)
    s = gpu_solver(A, cfg)
    x, info = s.solve(dev(b))
    x = x.cpu().numpy()
    assert info.status == 0 and io.status == 0
    assert info.rel_res_true <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    # same algorithm, same hierarchy: the iterates agree to rounding, in norm
    # and entry by entry
    assert np.linalg.norm(x - xo) <= 1e-7 * np.linalg.norm(xo)
    assert np.abs(x - xo).max() <= 1e-7 * np.abs(xo).max()
    # against a tight oracle solve (the reference solution)
    xt, _ = O.Hierarchy(A, dict(ocfg(cfg), rtol=1e-13)).solve(b)
    assert np.linalg.norm(x - xt) <= 1e-7 * np.linalg.norm(xt)
    assert np.abs(x - xt).max() <= max(2.0 * np.abs(xo - xt).max(), 1e-7 * np.abs(xt).max())


@pytest.mark.parametrize("name", ["poisson2d_64", "grf3d_24", "convdiff_14", "grf3d_33", "poisson2d_181",
                                  "convdiff_29", "grf3d_61"])
def test_vcycle_parity(name):
    A = SMALL_CASES[name]()
    r = np.random.default_rng(1).uniform(-1, 1, A.n)
    zo = O.Hierarchy(A).vcycle(r)
    z = gpu_solver(A).vcycle(dev(r)).cpu().numpy()
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)


@pytest.mark.parametrize("name", ["poisson2d_64", "grf3d_24", "grf3d_33", "grf3d_61"])
def test_vcycle_mixed_close_to_fp64(name):
    A = SMALL_CASES[name]()
    r = np.random.default_rng(1).uniform(-1, 1, A.n)
    zo = O.Hierarchy(A).vcycle(r)
    z = gpu_solver(A, {"precision": "MIXED"}).vcycle(dev(r)).cpu().numpy()
    assert np.linalg.norm(z - zo) <= 1e-5 * np.linalg.norm(zo)


@pytest.mark.parametrize("name,cfg", [("poisson2d_64", {}), ("grf3d_24", {}), ("logk2d_48", {}),
                                      ("convdiff_14", {"solver": "BICGSTAB"}), ("grf3d_61", {}),
                                      ("convdiff_29", {"solver": "BICGSTAB"})])
def test_mixed_precision_solve(name, cfg):
    A = SMALL_CASES[name]()
    b = np.random.default_rng(9).uniform(-1, 1, A.n)
    xo, io = O.Hierarchy(A, ocfg(cfg)).solve(b)
    xt, _ = O.Hierarchy(A, dict(ocfg(cfg), rtol=1e-13)).solve(b)
    s = gpu_solver(A, dict(cfg, precision="MIXED"))
    x, info = s.solve(dev(b))
    x = x.cpu().numpy()
    assert info.status == 0 and info.rel_res_true <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    assert np.linalg.norm(x - xt) <= 1e-7 * np.linalg.norm(xt)
    assert np.abs(x - xt).max() <= max(2.0 * np.abs(xo - xt).max(), 1e-7 * np.abs(xt).max())


@pytest.mark.parametrize("name,cfg", [("poisson2d_64", {}), ("logk2d_48", {}),
                                      ("convdiff_14", {"solver": "BICGSTAB"}),
                                      ("grf3d_24", {"precision": "MIXED"}),
                                      ("grf3d_33", {"precision": "MIXED"}),
                                      ("convdiff_29", {"solver": "BICGSTAB", "precision": "MIXED"})])
def test_adjoint_parity(name, cfg):
    A = SMALL_CASES[name]()
    rng = np.random.default_rng(3)
    b = rng.uniform(-1, 1, A.n)
    g = rng.uniform(-1, 1, A.n)
    ho = O.Hierarchy(A, dict(ocfg(cfg), rtol=1e-13))
    xo, _ = ho.solve(b)
    lam_o, dA_o, _ = ho.adjoint(xo, g, A.nnz)
    s = gpu_solver(A, cfg)
    x, _ = s.solve(dev(b))
    lam, dA, info = s.adjoint(x, dev(g))
    assert info.status == 0 and info.rel_res_true <= 1e-8
    lam = lam.cpu().numpy()
    dA = dA.cpu().numpy()
    assert np.linalg.norm(lam - lam_o) <= 1e-6 * np.linalg.norm(lam_o)
    assert np.linalg.norm(dA - dA_o) <= 1e-6 * np.linalg.norm(dA_o)
    assert np.abs(lam - lam_o).max() <= 1e-6 * np.abs(lam_o).max()
    assert np.abs(dA - dA_o).max() <= 1e-6 * np.abs(dA_o).max()
    # the stored-pattern product: exact given the GPU's own lambda and x
    rows = A.row_of()
    ref = -lam[rows] * x.cpu().numpy()[A.col_idx]
    assert np.array_equal(dA, ref)


def test_host_pointers_match_device():
    A = M.poisson2d(40)
    b = np.random.default_rng(2).uniform(-1, 1, A.n)
    s_host = api.Solver(A.row_ptr, A.col_idx, A.values)
    x_host, info_h = s_host.solve(b)
    x_dev, info_d = gpu_solver(A).solve(dev(b))
    assert isinstance(x_host, np.ndarray)
    assert np.array_equal(x_host, x_dev.cpu().numpy()) and info_h.iters == info_d.iters
    lam, dA, _ = s_host.adjoint(x_host, b)
    lam2, dA2, _ = gpu_solver(A).adjoint(dev(x_host), dev(b))
    assert np.array_equal(lam, lam2.cpu().numpy()) and np.array_equal(dA, dA2.cpu().numpy())


def test_adjoint_x_may_share_an_output_buffer():
    """x read in place by the gradient must not be the lambda buffer the
    adjoint fills first: such a call keeps a private copy of x."""
    A = M.diffusion3d_grf(N=16).A
    s = gpu_solver(A)
    rng = np.random.default_rng(12)
    x, _ = s.solve(dev(rng.uniform(-1, 1, A.n)))
    g = dev(rng.uniform(-1, 1, A.n))
    lam_ref, dA_ref, _ = s.adjoint(x, g)
    xa = x.clone()
    lam, dA, _ = s.adjoint(xa, g, lam=xa)
    assert lam.data_ptr() == xa.data_ptr()
    assert torch.equal(lam, lam_ref) and torch.equal(dA, dA_ref)


def test_host_pointers_nonsymmetric_adjoint():
    A = M.convdiff3d_upwind(N=14).A
    rng = np.random.default_rng(8)
    b, g = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    s_host = api.Solver(A.row_ptr, A.col_idx, A.values, {"solver": "BICGSTAB"})
    x_host, _ = s_host.solve(b)
    lam, dA, info = s_host.adjoint(x_host, g)
    assert info.status == 0
    lam2, dA2, _ = gpu_solver(A, {"solver": "BICGSTAB"}).adjoint(dev(x_host), dev(g))
    assert np.array_equal(lam, lam2.cpu().numpy()) and np.array_equal(dA, dA2.cpu().numpy())


def test_repeated_solves_are_deterministic():
    A = M.diffusion3d_grf(N=20).A
    s = gpu_solver(A)
    b = dev(np.random.default_rng(0).uniform(-1, 1, A.n))
    x1, i1 = s.solve(b)
    x2, i2 = s.solve(b)
    assert torch.equal(x1, x2) and i1.iters == i2.iters


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------

def test_single_level_dense():
    A = M.poisson2d(7)  # 49 rows: the coarsest level is the matrix itself
    b = np.random.default_rng(1).uniform(-1, 1, A.n)
    s = gpu_solver(A)
    assert s.info().nlevels == 1
    x, info = s.solve(dev(b))
    assert info.status == 0 and info.iters <= 2
    assert np.allclose(x.cpu().numpy(), np.linalg.solve(A.to_dense(), b), rtol=1e-10, atol=1e-12)


def test_one_by_one():
    A = M.CSR(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    x, info = gpu_solver(A).solve(dev(np.array([2.0])))
    assert info.status == 0 and x.item() == 0.5


def test_zero_rhs_and_nan_rhs():
    A = M.poisson2d(20)
    s = gpu_solver(A)
    x, info = s.solve(dev(np.zeros(A.n)))
    assert info.status == 0 and info.iters == 0 and not x.any()
    b = np.ones(A.n)
    b[7] = np.nan
    x, info = s.solve(dev(b))
    assert info.status == _lib.AMG_NAN


def test_maxit_status():
    A = M.poisson2d(30)
    s = gpu_solver(A, {"max_iter": 2, "max_restarts": 0})
    x, info = s.solve(dev(np.random.default_rng(0).uniform(-1, 1, A.n)))
    assert info.status == _lib.AMG_MAXIT and info.iters == 2


def test_invalid_csr_codes():
    A = M.poisson2d(6)
    bad = A.col_idx.copy()
    bad[0], bad[1] = bad[1], bad[0]
    with pytest.raises(api.AMGError) as e:
        api.Solver(dev(A.row_ptr), dev(bad), dev(A.values))
    assert e.value.code == _lib.AMG_ERR_BAD_CSR
    dpos = [k for k in range(A.row_ptr[3], A.row_ptr[4]) if A.col_idx[k] == 3][0]
    v = A.values.copy()
    v[dpos] = 0.0
    with pytest.raises(api.AMGError) as e:
        api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(v))
    assert e.value.code == _lib.AMG_ERR_ZERO_DIAG
    oob = A.col_idx.copy()
    oob[-1] = A.n + 5
    with pytest.raises(api.AMGError) as e:
        api.Solver(dev(A.row_ptr), dev(oob), dev(A.values))
    assert e.value.code == _lib.AMG_ERR_BAD_CSR
    rp = A.row_ptr.copy()
    rp[-1] += 1
    with pytest.raises(api.AMGError) as e:
        api.Solver(dev(rp), dev(A.col_idx), dev(A.values))
    assert e.value.code in (_lib.AMG_ERR_BAD_CSR, _lib.AMG_ERR_ARG)


def test_empty_row_is_missing_diagonal():
    rp = np.array([0, 2, 2, 4], np.int32)  # row 1 stores nothing (nnz >= n still)
    ci = np.array([0, 2, 0, 2], np.int32)
    v = np.array([1.0, 0.5, 0.5, 1.0])
    with pytest.raises(api.AMGError) as e:
        api.Solver(dev(rp), dev(ci), dev(v))
    assert e.value.code == _lib.AMG_ERR_ZERO_DIAG


def test_not_spd_declared_symmetric():
    D = np.array([[1.0, 2.0], [2.0, 1.0]])
    A = M.CSR(np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), D.reshape(-1).copy())
    with pytest.raises(api.AMGError) as e:
        gpu_solver(A, {"symmetric": 1})
    assert e.value.code == _lib.AMG_NOT_SPD


def test_symmetry_detection_and_nonsymmetric_adjoint_reuse():
    A = M.convdiff3d_upwind(N=10).A
    s = gpu_solver(A, {"solver": "BICGSTAB"})
    b = dev(np.ones(A.n))
    x, _ = s.solve(b)
    lam1, _, i1 = s.adjoint(x, b)
    lam2, _, i2 = s.adjoint(x, b)  # second call reuses the cached A^T hierarchy
    assert torch.equal(lam1, lam2)
    At = A.to_dense().T
    assert np.allclose(lam1.cpu().numpy(), np.linalg.solve(At, np.ones(A.n)), rtol=1e-7, atol=1e-10)


# ---------------------------------------------------------------------------
# Full-size workloads in the launch configuration bench.py times
# ---------------------------------------------------------------------------

@pytest.mark.slow
@pytest.mark.parametrize("gen,cfg", [
    (lambda: M.diffusion3d_grf(N=128), {"solver": "PCG"}),
    (lambda: M.convdiff3d_upwind(N=160), {"solver": "BICGSTAB"}),
])
def test_full_size_parity(gen, cfg):
    """128^3 GRF diffusion and 160^3 convection-diffusion, in the launch
    configuration the benchmark times: the aggregates of every level and
    every coarse operator (pattern and values) bit-exact in both precision
    forms.  Their solutions and gradients are held to the oracle in
    test_gpu_error_bars.py."""
    w = gen()
    A = w.A
    h = O.Hierarchy(A, ocfg(cfg))
    for prec in ("FP64", "MIXED"):
        s = gpu_solver(A, dict(cfg, precision=prec))
        info = s.info()
        assert info.nlevels == h.nlevels
        for l in range(h.nlevels - 1):
            lv, nxt = h.level(l), h.level(l + 1)
            assert np.array_equal(s.aggregates(l), lv.agg), (prec, l)
            for which, ref in (("P", lv.P), ("R", lv.R), ("A", None)):
                ref = ref if ref is not None else nxt.A
                rp, ci, v, _ = s.level(l if which != "A" else l + 1, which)
                assert np.array_equal(rp, ref.row_ptr) and np.array_equal(ci, ref.col_idx), (prec, which, l)
                assert np.array_equal(v.view(np.int64), ref.values.view(np.int64)), (prec, which, l)
        s.close()


# ---------------------------------------------------------------------------
# BiCGStab breakdown and its one restart
# ---------------------------------------------------------------------------

def _dense_csr(D):
    rows, cols = np.nonzero(D)
    rp = np.zeros(D.shape[0] + 1, np.int32)
    rp[1:] = np.cumsum(np.bincount(rows, minlength=D.shape[0]))
    return M.CSR(rp, cols.astype(np.int32), D[rows, cols].astype(np.float64))


def test_bicgstab_breakdown_restart_parity():
    """rho = r^.r is exactly 0 at iteration 2 of this dyadic system (see the
    oracle's pin): the GPU restarts once from x with r^ = r, as the oracle
    does, and converges to A^-1 b in the same iterations."""
    D = np.array([[3.0, 0.0, 3.0], [0.0, 4.0, -1.0], [1.0, 0.0, 2.0]])
    A = _dense_csr(D)
    b = np.ones(3)
    cfg = {"solver": "BICGSTAB_NOPREC", "rtol": 1e-12}
    xo, io = O.solve(A, b, ocfg(cfg))
    x, info = gpu_solver(A, cfg).solve(dev(b))
    assert io.status == O.OK and info.status == 0, info
    assert info.iters == io.iters == 3
    assert np.allclose(x.cpu().numpy(), np.linalg.solve(D, b), rtol=0, atol=1e-14)


def test_bicgstab_second_breakdown_status():
    """r^.A b = 0 at the first iteration and again after the one restart:
    BREAKDOWN after two iterations, x still 0, as in the oracle."""
    D = np.array([[1.0, -2.0], [0.0, 1.0]])
    A = _dense_csr(D)
    cfg = {"solver": "BICGSTAB_NOPREC"}
    xo, io = O.solve(A, np.ones(2), ocfg(cfg))
    x, info = gpu_solver(A, cfg).solve(dev(np.ones(2)))
    assert io.status == O.BREAKDOWN and info.status == _lib.AMG_BREAKDOWN
    assert info.iters == io.iters == 2
    assert not x.cpu().numpy().any()


def test_profile_product_leaves_the_handle_ready():
    """amg_profile_product times the Krylov product on the last solve's
    vectors and leaves the handle as it found it: the next solve gives the
    same bits."""
    A = M.diffusion3d_grf(N=33).A
    b = dev(np.random.default_rng(4).uniform(-1, 1, A.n))
    for cfg in ({}, {"precision": "MIXED"}):
        s = gpu_solver(A, cfg)
        x1, i1 = s.solve(b)
        us = s.profile_product(5)
        assert 0.0 < us < 1e4
        x2, i2 = s.solve(b)
        assert torch.equal(x1, x2) and i1.iters == i2.iters
    s = gpu_solver(M.convdiff3d_upwind(N=14).A, {"solver": "BICGSTAB"})
    s.solve(dev(np.ones(14 ** 3)))
    assert s.profile_product(3) > 0.0


@pytest.mark.parametrize("cfg", [{}, {"precision": "MIXED"}, {"solver": "BICGSTAB"}, {"solver": "CG"}])
def test_device_loop_matches_host_polled_loop(cfg):
    """The device-side Krylov loop (a conditional graph node) and the
    host-polled graphs run the same iterations: same bits, same counts."""
    A = M.diffusion3d_grf(N=24).A if cfg.get("solver") != "BICGSTAB" else M.convdiff3d_upwind(N=14).A
    b = dev(np.random.default_rng(6).uniform(-1, 1, A.n))
    out = []
    for loop in (1, 0):
        s = gpu_solver(A, dict(cfg, device_loop=loop, max_iter=2000))
        x, info = s.solve(b)
        assert info.status == 0
        out.append((x, info.iters))
        s.close()
    assert torch.equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
