"""GPU parity of the whole PCG solve in one cluster launch (csrc/cpcg.cuh).

Where every level's operators fit one cluster's shared memory, a PCG solve
(Sec. 2.1) runs its iterations in a single launch: the V-cycle, q = A p and
the updates exchange vectors through distributed shared memory, and the dot
products are summed in rank order in every CTA.  Its results are held to the
FP64 oracle at the same bars as every other solve (x, lambda and dA within
1e-7 of the oracle's, in norm and entry by entry), and to the per-iteration
kernels of the host-polled loop (device_loop = 0): the same iterations up to
the dot products' summation order."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_09001_b300 import _lib, api, matrices as M

pytestmark = pytest.mark.gpu

# 4096 -> 585 -> dense 51; 3000-row tridiagonal; 16^3 diffusion (4096 rows,
# 3D stencil); a log-normal 2D field (4900 rows)
CASES = {
    "poisson2d_64": lambda: M.poisson2d(64),
    "tri_3000": lambda: M.tridiagonal_matrix(3000),
    "grf3d_16": lambda: M.diffusion3d_grf(N=16).A,
    "logk2d_70": lambda: M.diffusion2d_logk(N=70).A,
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def solver(A, cfg=None):
    return api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values), cfg or {})


def launched(s, fn, levels=False):
    """Names of the traced launches of fn() (with levels: (name, level) pairs)."""
    s.profile(True)
    fn()
    _, recs = s.profile_records()
    s.profile(False)
    if levels:
        return {(r["name"], r["level"]) for r in recs if r["launches"] > 0}
    return {r["name"] for r in recs if r["launches"] > 0}


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("name", list(CASES))
def test_cluster_solve_matches_oracle_and_host_loop(name, precision):
    A = CASES[name]()
    b = np.random.default_rng(7).uniform(-1, 1, A.n)
    s = solver(A, {"precision": precision})
    names = launched(s, lambda: s.solve(dev(b)))
    assert "cluster_pcg" in names and "pcg_update" not in names, names
    x, info = s.solve(dev(b))
    x = x.cpu().numpy()
    assert info.status == 0 and info.rel_res_true <= 1e-8
    # deterministic: a second solve gives the same bits
    x2, info2 = s.solve(dev(b))
    assert same_bits(x2.cpu().numpy(), x) and info2.iters == info.iters
    # the oracle
    xo, io = O.Hierarchy(A).solve(b)
    xt, _ = O.Hierarchy(A, {"rtol": 1e-13}).solve(b)
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    assert np.linalg.norm(x - xt) <= 1e-7 * np.linalg.norm(xt)
    assert np.abs(x - xt).max() <= max(2.0 * np.abs(xo - xt).max(), 1e-7 * np.abs(xt).max())
    # the per-iteration kernels
    h = solver(A, {"precision": precision, "device_loop": 0})
    assert "cluster_pcg" not in launched(h, lambda: h.solve(dev(b)))
    xh, ih = h.solve(dev(b))
    xh = xh.cpu().numpy()
    assert ih.status == 0 and abs(ih.iters - info.iters) <= 1, (ih.iters, info.iters)
    assert np.linalg.norm(x - xh) <= 1e-7 * np.linalg.norm(xh)


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("name", ["poisson2d_64", "logk2d_70"])
def test_cluster_adjoint_matches_oracle(name, precision):
    A = CASES[name]()
    rng = np.random.default_rng(3)
    b, g = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    ho = O.Hierarchy(A, {"rtol": 1e-13})
    xo, _ = ho.solve(b)
    lam_o, dA_o, _ = ho.adjoint(xo, g, A.nnz)
    s = solver(A, {"precision": precision})
    x, _ = s.solve(dev(b))
    names = launched(s, lambda: s.adjoint(x, dev(g)))
    assert "cluster_pcg" in names, names
    lam, dA, info = s.adjoint(x, dev(g))
    assert info.status == 0 and info.rel_res_true <= 1e-8
    lam, dA = lam.cpu().numpy(), dA.cpu().numpy()
    for got, ref in ((lam, lam_o), (dA, dA_o)):
        assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref)
        assert np.abs(got - ref).max() <= 1e-7 * np.abs(ref).max()
    assert np.array_equal(dA, -lam[A.row_of()] * x.cpu().numpy()[A.col_idx])


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_cluster_iteration_cap(precision):
    """max_iter ends the launch with MAXIT after exactly max_iter iterations,
    as the per-iteration loop does.  After four iterations the iterates still
    carry the preconditioner's rounding: FP64 cycles agree to 1e-10; the two
    mixed paths apply FP32 cycles rounded differently (the cluster launch the
    collapsed coarse end's FP32 copy with FP32 sums), so 1e-6."""
    A = CASES["poisson2d_64"]()
    b = np.random.default_rng(2).uniform(-1, 1, A.n)
    res = []
    for loop in (1, 0):
        s = solver(A, {"precision": precision, "max_iter": 4, "device_loop": loop})
        x, info = s.solve(dev(b))
        assert info.status == _lib.AMG_MAXIT and info.iters == 4, (info.status, info.iters)
        res.append(x.cpu().numpy())
    tol = 1e-10 if precision == "FP64" else 1e-6
    assert np.linalg.norm(res[0] - res[1]) <= tol * np.linalg.norm(res[1])


def test_cluster_zero_and_nan_right_hand_sides():
    A = CASES["tri_3000"]()
    s = solver(A)
    x, info = s.solve(dev(np.zeros(A.n)))
    assert info.status == 0 and info.iters == 0 and not x.cpu().numpy().any()
    b = np.random.default_rng(1).uniform(-1, 1, A.n)
    b[17] = np.nan
    _, info = s.solve(dev(b))
    assert info.status == _lib.AMG_NAN
    # the handle stays usable
    b[17] = 0.5
    x, info = s.solve(dev(b))
    assert info.status == 0 and info.rel_res_true <= 1e-8


def test_cluster_tight_tolerance_restarts_from_the_true_residual():
    """rtol 1e-13: the recursion may meet the tolerance before the true
    residual does; the host restarts the launch from x and b - A x, and the
    result is held to the oracle."""
    A = CASES["logk2d_70"]()
    b = np.random.default_rng(4).uniform(-1, 1, A.n)
    s = solver(A, {"rtol": 1e-13, "max_iter": 400})
    x, info = s.solve(dev(b))
    assert info.status in (0, _lib.AMG_MAXIT)
    if info.status == 0:
        assert info.rel_res_true <= 1e-13
    xt, _ = O.Hierarchy(A, {"rtol": 1e-13}).solve(b)
    assert np.linalg.norm(x.cpu().numpy() - xt) <= 1e-9 * np.linalg.norm(xt)


@pytest.mark.parametrize("case", ["bicgstab", "host_loop", "large", "fuse0"])
def test_cluster_solve_not_taken(case):
    A, cfg = {
        "bicgstab": (CASES["poisson2d_64"], {"solver": "BICGSTAB"}),
        "host_loop": (CASES["poisson2d_64"], {"device_loop": 0}),
        # 40000 rows: the finest level streams
        "large": (lambda: M.poisson2d(200), {}),
        "fuse0": (CASES["poisson2d_64"], {"fuse_coarse": 0}),
    }[case]
    A = A()
    b = np.random.default_rng(8).uniform(-1, 1, A.n)
    s = solver(A, cfg)
    assert "cluster_pcg" not in launched(s, lambda: s.solve(dev(b)))
    x, info = s.solve(dev(b))
    assert info.status == 0 and info.rel_res_true <= 1e-8


# tails that start below the finest level: 32,761 rows (streamed) -> 4,648 ->
# dense 427; the cluster kernel runs the cycle from level 1 (V-cycle mode)
CYCLE_CASES = {
    "logk2d_181": lambda: M.diffusion2d_logk(N=181).A,
    "poisson2d_181": lambda: M.poisson2d(181),
}


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("name", list(CYCLE_CASES))
def test_cluster_cycle_from_a_coarse_level(name, precision):
    A = CYCLE_CASES[name]()
    rng = np.random.default_rng(21)
    r = rng.uniform(-1, 1, A.n)
    s = solver(A, {"precision": precision})
    runs = launched(s, lambda: s.vcycle(dev(r)), levels=True)
    names = {n for n, _ in runs}
    assert "cluster_cycle" in names and "tail" not in names, names
    # the launch restricts into its first level t itself: no restriction pass
    # from level t-1 runs
    (t,) = [lv for n, lv in runs if n == "cluster_cycle"]
    assert t >= 1 and ("restrict", t - 1) not in runs and ("presmooth", t - 1) in runs, runs
    z = s.vcycle(dev(r)).cpu().numpy()
    zo = O.Hierarchy(A).vcycle(r)
    tol = 1e-12 if precision == "FP64" else 1e-5
    assert np.linalg.norm(z - zo) <= tol * np.linalg.norm(zo)
    # the per-pass cycle of the same hierarchy (fuse_coarse = 0)
    p = solver(A, {"precision": precision, "fuse_coarse": 0})
    zp = p.vcycle(dev(r)).cpu().numpy()
    assert np.linalg.norm(z - zp) <= tol * np.linalg.norm(zp)
    # solve and adjoint against the oracle
    b, g = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    ho = O.Hierarchy(A, {"rtol": 1e-13})
    xt, _ = ho.solve(b)
    lam_t, _, _ = ho.adjoint(xt, g, A.nnz)
    x, info = s.solve(dev(b))
    assert info.status == 0 and info.rel_res_true <= 1e-8
    lam, _, ainfo = s.adjoint(x, dev(g))
    assert ainfo.status == 0
    x, lam = x.cpu().numpy(), lam.cpu().numpy()
    assert np.linalg.norm(x - xt) <= 1e-7 * np.linalg.norm(xt)
    assert np.abs(x - xt).max() <= 1e-7 * np.abs(xt).max()
    assert np.linalg.norm(lam - lam_t) <= 1e-7 * np.linalg.norm(lam_t)
