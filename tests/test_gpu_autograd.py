"""The adjoint behind torch.autograd (Sec. 2.1 "JAX integration", Eq. 1-2):
gradients of a loss through the GPU solve, with respect to per-cell
log-conductivities (through the differentiable FV assembly) and the
right-hand side, checked against central finite differences and against the
FP64 oracle's adjoint; and the paper's Sec. 3.2 inverse problem run end to
end on the GPU."""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M
from paper_2606_09001_b300.autograd import amg_solve
from paper_2606_09001_b300.fv_torch import fv_values

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")


def setup_problem(N, seed=2):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, 1.0, size=(N, N))
    b = rng.uniform(-1, 1, N * N)
    xt = rng.uniform(-1, 1, N * N)
    A = M.diffusion_fv(np.exp(theta))
    return theta, b, xt, A


def loss_and_grads(theta, b, xt, A, cfg, cache):
    dev = torch.device("cuda")
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    th = torch.tensor(theta, device=dev, requires_grad=True)
    bt = torch.tensor(b, device=dev, requires_grad=True)
    x = amg_solve(rp, ci, fv_values(th), bt, cfg, cache)
    L = ((x - torch.tensor(xt, device=dev)) ** 2).sum()
    L.backward()
    return L.item(), th.grad.cpu().numpy(), bt.grad.cpu().numpy()


def loss_only(theta, b, xt, A, cfg, cache):
    dev = torch.device("cuda")
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    with torch.no_grad():
        x = amg_solve(rp, ci, fv_values(torch.tensor(theta, device=dev)), torch.tensor(b, device=dev), cfg, cache)
        return float(((x - torch.tensor(xt, device=dev)) ** 2).sum())


def oracle_grads(theta, b, xt, A):
    """dL/dtheta and dL/db from the oracle's solve and adjoint (rtol 1e-13),
    chained through the same FV assembly on the CPU."""
    h = O.Hierarchy(A, {"rtol": 1e-13})
    x, _ = h.solve(b)
    lam, dA, _ = h.adjoint(x, 2 * (x - xt), A.nnz)
    th = torch.tensor(theta, requires_grad=True)
    fv_values(th).backward(torch.from_numpy(dA))
    return th.grad.numpy(), lam


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_autograd_matches_central_fd(prec):
    theta, b, xt, A = setup_problem(24)
    cfg = {"rtol": 1e-12, "precision": prec, "max_iter": 1000}
    cache = api.SetupCache()
    L0, gth, gb = loss_and_grads(theta, b, xt, A, cfg, cache)
    rng = np.random.default_rng(5)
    eps = 1e-5
    for _ in range(3):
        v = rng.normal(size=theta.shape)
        fd = (loss_only(theta + eps * v, b, xt, M.diffusion_fv(np.exp(theta + eps * v)), cfg, cache)
              - loss_only(theta - eps * v, b, xt, M.diffusion_fv(np.exp(theta - eps * v)), cfg, cache)) / (2 * eps)
        assert np.sum(gth * v) == pytest.approx(fd, rel=1e-5)
        u = rng.normal(size=b.shape)
        fdb = (loss_only(theta, b + eps * u, xt, A, cfg, cache) - loss_only(theta, b - eps * u, xt, A, cfg, cache)) / (2 * eps)
        assert np.sum(gb * u) == pytest.approx(fdb, rel=1e-5)
    cache.clear()


def test_autograd_matches_oracle_gradient():
    theta, b, xt, A = setup_problem(40)
    cache = api.SetupCache()
    _, gth, gb = loss_and_grads(theta, b, xt, A, {"rtol": 1e-12}, cache)
    gth_o, lam_o = oracle_grads(theta, b, xt, A)
    assert np.linalg.norm(gth - gth_o) <= 1e-6 * np.linalg.norm(gth_o)
    assert np.linalg.norm(gb - lam_o) <= 1e-6 * np.linalg.norm(lam_o)
    cache.clear()


def test_setup_cache_reuses_hierarchy_across_backward():
    theta, b, xt, A = setup_problem(20)
    cache = api.SetupCache()
    loss_and_grads(theta, b, xt, A, {"rtol": 1e-10}, cache)
    assert cache.misses == 1  # backward reused the forward hierarchy (symmetric A)
    loss_and_grads(theta, b, xt, A, {"rtol": 1e-10}, cache)
    assert cache.misses == 1 and cache.hits >= 1
    loss_and_grads(theta + 0.1, b, xt, A, {"rtol": 1e-10}, cache)
    assert cache.misses == 1 and cache.resetups == 1  # new values: numeric re-setup of the cached hierarchy
    cache.clear()
    fresh = api.SetupCache(resetup=False)
    loss_and_grads(theta, b, xt, A, {"rtol": 1e-10}, fresh)
    loss_and_grads(theta + 0.1, b, xt, A, {"rtol": 1e-10}, fresh)
    assert fresh.misses == 2 and fresh.resetups == 0  # without re-setup: a fresh setup
    fresh.clear()


def test_autograd_nonsymmetric_fd():
    A = M.convdiff3d_upwind(N=8).A
    rng = np.random.default_rng(3)
    b = rng.uniform(-1, 1, A.n)
    xt = rng.uniform(-1, 1, A.n)
    dev = torch.device("cuda")
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    cfg = {"solver": "BICGSTAB", "rtol": 1e-12}
    cache = api.SetupCache()

    def L(vals, grad=False):
        v = torch.tensor(vals, device=dev, requires_grad=grad)
        x = amg_solve(rp, ci, v, torch.tensor(b, device=dev), cfg, cache)
        out = ((x - torch.tensor(xt, device=dev)) ** 2).sum()
        if grad:
            out.backward()
            return out.item(), v.grad.cpu().numpy()
        return out.item()

    _, g = L(A.values, True)
    eps = 1e-5
    for _ in range(3):
        d = rng.normal(size=A.nnz)
        fd = (L(A.values + eps * d) - L(A.values - eps * d)) / (2 * eps)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-5)
    cache.clear()


def test_paper_example2_on_gpu():
    """Sec. 3.2: recover d of tridiag(-1, d, -1) from x(d = 4) by gradient
    descent from d = 10 with lr 0.1, gradients through the GPU adjoint."""
    g = json.load(open(GOLDEN))["ex2_tridiagonal_inverse"]
    n = g["n"]
    dev = torch.device("cuda")
    A = M.tridiagonal_matrix(n, g["true_diag"])
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    is_diag = torch.from_numpy(A.row_of() == A.col_idx).to(dev)
    b = torch.ones(n, dtype=torch.float64, device=dev)
    cfg = {"rtol": 1e-12}
    cache = api.SetupCache(capacity=2)

    def values(d):
        return torch.where(is_diag, d, torch.tensor(-1.0, dtype=torch.float64, device=dev))

    with torch.no_grad():
        x_t = amg_solve(rp, ci, values(torch.tensor(g["true_diag"], dtype=torch.float64, device=dev)), b, cfg, cache)
    d = torch.tensor(g["init_diag"], dtype=torch.float64, device=dev, requires_grad=True)
    d_at_bound = None
    for step in range(g["max_iters"]):
        x = amg_solve(rp, ci, values(d), b, cfg, cache)
        loss = ((x - x_t) ** 2).sum()
        (grad,) = torch.autograd.grad(loss, d)
        with torch.no_grad():
            d -= g["lr"] * grad
        if step + 1 == g["steps_upper_bound"]:
            d_at_bound = d.item()
        if abs(grad.item()) < g["grad_tol"]:
            break
    assert abs(d_at_bound - g["true_diag"]) < g["recover_abs_tol"]
    assert abs(d.item() - g["true_diag"]) < 1e-3
    cache.clear()


@pytest.mark.slow
def test_full_size_c3_gradient():
    """512^2 cells, log k ~ N(0,1): the mixed-precision GPU gradient at
    rtol 1e-8 within 1e-6 of the oracle's at rtol 1e-13 (measured: ~1e-8)."""
    w = M.diffusion2d_logk()
    theta, b, xt, A = w.extra["theta"], w.b, w.extra["x_target"], w.A
    cache = api.SetupCache()
    _, gth, gb = loss_and_grads(theta, b, xt, A, {"rtol": 1e-8, "precision": "MIXED"}, cache)
    gth_o, lam_o = oracle_grads(theta, b, xt, A)
    rel_t = np.linalg.norm(gth - gth_o) / np.linalg.norm(gth_o)
    rel_b = np.linalg.norm(gb - lam_o) / np.linalg.norm(lam_o)
    print(f"C3 512^2: gradient error vs oracle {rel_t:.2e} (theta), {rel_b:.2e} (b)")
    assert rel_t <= 1e-6 and rel_b <= 1e-6
    cache.clear()
