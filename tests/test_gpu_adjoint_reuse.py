"""GPU parity of the nonsymmetric adjoint with transposed-hierarchy reuse
(amg_config.adjoint_reuse = 1): the adjoint solve runs on A's aggregates and
prolongators with every level operator transposed, against the oracle's
transposed hierarchy (or_transposed), before and after a numeric re-setup."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg  # noqa: F401  (sp.linalg)
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M

pytestmark = pytest.mark.gpu

DEV = "cuda"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def solver(A, cfg):
    return api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values), cfg)


CASES = {
    "convdiff_14": lambda: M.convection_diffusion_upwind(14),
    # streaming kernels on level 0 (24,389 rows)
    "convdiff_29": lambda: M.convection_diffusion_upwind(29),
}


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_reuse_matches_oracle(name, precision):
    A = CASES[name]()
    rng = np.random.default_rng(11)
    b, g = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    ho = O.Hierarchy(A, {"solver": 1, "adjoint_reuse": 1})
    xo, _ = ho.solve(b)
    _, _, aio = ho.adjoint(xo, g, A.nnz)
    ht = O.Hierarchy(A, {"solver": 1, "adjoint_reuse": 1, "rtol": 1e-13})
    xt, _ = ht.solve(b)
    lam_t, _, _ = ht.adjoint(xt, g, A.nnz)
    s = solver(A, {"solver": "BICGSTAB", "adjoint_reuse": 1, "precision": precision})
    x, info = s.solve(dev(b))
    lam, dA, ainfo = s.adjoint(x, dev(g))
    assert info.status == 0 and ainfo.status == 0 and ainfo.rel_res_true <= 1e-8
    assert abs(ainfo.iters - aio.iters) <= 2, (ainfo.iters, aio.iters)
    lam = lam.cpu().numpy()
    assert np.linalg.norm(lam - lam_t) <= 1e-6 * np.linalg.norm(lam_t)
    rows = A.row_of()
    assert np.array_equal(dA.cpu().numpy(), -lam[rows] * x.cpu().numpy()[A.col_idx])
    At = sp.csr_matrix((A.values, A.col_idx, A.row_ptr), shape=(A.n, A.n)).T.tocsr()
    assert np.linalg.norm(At @ lam - g) <= 1e-8 * np.linalg.norm(g) * 1.0001


def test_adjoint_reuse_follows_a_resetup():
    """After new values on the pattern, the transposed hierarchy is refreshed
    from the re-set-up forward one: the adjoint matches the oracle's
    transposed hierarchy of the oracle's re-setup."""
    A0 = M.convection_diffusion_upwind(29)
    rng = np.random.default_rng(12)
    A1 = M.CSR(A0.row_ptr, A0.col_idx, A0.values * rng.uniform(0.8, 1.25, A0.nnz))
    b, g = rng.uniform(-1, 1, A0.n), rng.uniform(-1, 1, A0.n)
    s = solver(A0, {"solver": "BICGSTAB", "adjoint_reuse": 1})
    x0, _ = s.solve(dev(b))
    s.adjoint(x0, dev(g))  # builds the transposed hierarchy
    s.resetup(dev(A1.values))
    x, _ = s.solve(dev(b))
    lam, _, ainfo = s.adjoint(x, dev(g))
    cfg = {"solver": 1, "adjoint_reuse": 1}
    hr = O.Hierarchy(A0, cfg).resetup(A1.values)
    xo, _ = hr.solve(b)
    _, _, aio = hr.adjoint(xo, g, A1.nnz)
    assert ainfo.status == 0 and ainfo.rel_res_true <= 1e-8
    assert abs(ainfo.iters - aio.iters) <= 2, (ainfo.iters, aio.iters)
    At = sp.csr_matrix((A1.values, A1.col_idx, A1.row_ptr), shape=(A1.n, A1.n)).T.tocsr()
    lam = lam.cpu().numpy()
    lam_ref = sp.linalg.spsolve(At.tocsc(), g)
    assert np.linalg.norm(lam - lam_ref) <= 1e-6 * np.linalg.norm(lam_ref)


def test_adjoint_reuse_is_validated_and_symmetric_unaffected():
    A = M.poisson2d(40)
    with pytest.raises(api.AMGError):
        solver(A, {"adjoint_reuse": 2})
    b = dev(np.random.default_rng(3).uniform(-1, 1, A.n))
    s0, s1 = solver(A, {}), solver(A, {"adjoint_reuse": 1})
    x, _ = s0.solve(b)
    l0, _, _ = s0.adjoint(x, b)
    l1, _, _ = s1.adjoint(x, b)
    assert torch.equal(l0, l1)  # symmetric: the forward hierarchy either way
