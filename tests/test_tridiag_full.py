"""The tridiagonal system of Sec. 3.2 and Sec. 4 (tridiag(-1, 4, -1), b = ones)
at its full size n = 10^7, in the configuration bench.py times (unpreconditioned
CG, FP64; unpreconditioned BiCGStab as well, the paper's other Krylov method on
it).

The system has a closed-form solution.  With t = 2 - sqrt(3), the smaller root
of t^2 - 4 t + 1 = 0, the homogeneous solutions of the interior rows are t^i
and t^-i; adding the particular solution 1/2 and imposing x_0 = x_{n+1} = 0
gives x_i = (1 - (t^i + t^(n+1-i)) / (1 + t^(n+1))) / 2 for i = 1..n.  The CPU
test pins that formula (dense solve, the oracle's CG); the GPU test compares
the full-size solve with it.  The condition number of A is below 3 (spectrum
in (2, 6)), so a true residual of 1e-8 bounds the relative error by 3e-8.
The adjoint is checked through an independent residual of A^T lambda = g and
dL/dA = -lambda_i x_j on every stored entry, bit for bit."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M


def closed_form(n: int) -> np.ndarray:
    t = 2.0 - np.sqrt(3.0)
    i = np.arange(1, n + 1, dtype=np.float64)
    with np.errstate(under="ignore"):
        tn1 = t ** (n + 1)
        return 0.5 * (1.0 - (t ** i + t ** (n + 1 - i)) / (1.0 + tn1))


def tridiag_apply(x: np.ndarray, d: float = 4.0) -> np.ndarray:
    """A x for tridiag(-1, d, -1), written with shifted slices (no CSR)."""
    y = d * x
    y[1:] -= x[:-1]
    y[:-1] -= x[1:]
    return y


def test_closed_form_is_pinned():
    n = 60
    A = M.tridiagonal_matrix(n, 4.0).to_dense()
    xs = np.linalg.solve(A, np.ones(n))
    assert np.allclose(closed_form(n), xs, rtol=1e-14, atol=1e-15)
    n = 3000
    x, info = O.solve(M.tridiagonal_matrix(n, 4.0), np.ones(n), {"solver": 2, "rtol": 1e-12})
    assert info.status == 0
    assert np.linalg.norm(x - closed_form(n)) <= 1e-11 * np.linalg.norm(closed_form(n))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("solver_name", ["CG", "BICGSTAB_NOPREC"])
def test_full_size_tridiagonal(solver_name):
    w = M.tridiagonal_1e7()
    A, n = w.A, w.A.n
    s = api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values), {"solver": solver_name})
    x, info = s.solve(dev(w.b))
    assert info.status == 0 and info.rel_res_true <= 1e-8, info
    xn = x.cpu().numpy()
    xs = closed_form(n)
    assert np.linalg.norm(xn - xs) <= 3e-8 * np.linalg.norm(xs)
    assert np.linalg.norm(w.b - tridiag_apply(xn)) <= 1e-8 * np.linalg.norm(w.b)
    g = np.random.default_rng(17).uniform(-1, 1, n)
    lam, dA, ainfo = s.adjoint(x, dev(g))
    assert ainfo.status == 0 and ainfo.rel_res_true <= 1e-8, ainfo
    lam = lam.cpu().numpy()
    # A is symmetric: A^T lambda = A lambda
    assert np.linalg.norm(g - tridiag_apply(lam)) <= 1e-8 * np.linalg.norm(g)
    rows = A.row_of()
    assert np.array_equal(dA.cpu().numpy(), -lam[rows] * xn[A.col_idx])
    s.close()
