"""GPU parity of the mixed form's double-FP32 Krylov product.

In the mixed form the outer product q = A p of a streamed finest level may run
in double-FP32 arithmetic (amg_config.outer_product: -1 chosen at setup by
timing, 0 FP64, 1 double-FP32): A's values and p are pairs of binary32
numbers, and each product and row sum is accurate to a few 2^-48 of
sum_j |a_ij p_j|.  Both forced settings are held to the FP64 oracle at the
bars of every other solve (x, lambda, dA within 1e-7, in norm and entry by
entry), run the same number of iterations within one, and agree with each
other to far below the solve's tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M

pytestmark = pytest.mark.gpu

# finest levels that stream (>= 16384 rows), with the sliced-ELL layout (a
# ring of tiles) and the direct sliced-ELL layout for the product
CASES = {
    "grf3d_61": lambda: M.diffusion3d_grf(N=61).A,      # 226,981 rows, 3D 7-point
    "logk2d_181": lambda: M.diffusion2d_logk(N=181).A,  # 32,761 rows, 2D 5-point
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def solver(A, cfg):
    return api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values), cfg)


@pytest.mark.parametrize("layout", ["SLICED_ELL", "ELL_DIRECT"])
@pytest.mark.parametrize("name", list(CASES))
def test_df_product_solve_and_adjoint_match_oracle(name, layout):
    A = CASES[name]()
    rng = np.random.default_rng(13)
    b, g = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    ho = O.Hierarchy(A, {"rtol": 1e-13})
    xt, _ = ho.solve(b)
    lam_t, dA_t, _ = ho.adjoint(xt, g, A.nnz)
    xo, io = O.Hierarchy(A).solve(b)
    res = {}
    for df in (0, 1):
        s = solver(A, {"precision": "MIXED", "layout": layout, "outer_product": df})
        p = s.plan(0, "krylov")
        assert p["layout"] == layout and p["df"] == bool(df), p
        x, info = s.solve(dev(b))
        assert info.status == 0 and info.rel_res_true <= 1e-8
        assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
        lam, dA, ainfo = s.adjoint(x, dev(g))
        assert ainfo.status == 0 and ainfo.rel_res_true <= 1e-8
        x, lam, dA = x.cpu().numpy(), lam.cpu().numpy(), dA.cpu().numpy()
        assert np.linalg.norm(x - xt) <= 1e-7 * np.linalg.norm(xt)
        assert np.abs(x - xt).max() <= max(2.0 * np.abs(xo - xt).max(), 1e-7 * np.abs(xt).max())
        for got, ref in ((lam, lam_t), (dA, dA_t)):
            assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref)
        res[df] = (x, info.iters)
        s.close()
    (x0, i0), (x1, i1) = res[0], res[1]
    assert abs(i0 - i1) <= 1
    assert np.linalg.norm(x1 - x0) <= 1e-8 * np.linalg.norm(x0)


def test_df_product_follows_the_setting():
    A = CASES["grf3d_61"]()
    b = dev(np.random.default_rng(2).uniform(-1, 1, A.n))
    for cfg, want in (({"precision": "FP64", "outer_product": 1}, False),
                      ({"precision": "MIXED", "outer_product": 0}, False),
                      ({"precision": "MIXED", "outer_product": 1, "layout": "SLICED_ELL"}, True)):
        with solver(A, cfg) as s:
            assert s.plan(0, "krylov")["df"] == want, cfg
            _, info = s.solve(b)
            assert info.status == 0 and info.rel_res_true <= 1e-8
    # automatic: either choice, a correct solve
    with solver(A, {"precision": "MIXED"}) as s:
        assert isinstance(s.plan(0, "krylov")["df"], bool)
        _, info = s.solve(b)
        assert info.status == 0 and info.rel_res_true <= 1e-8


def test_df_product_resetup_refreshes_the_split_values():
    """A re-setup recomputes the double-FP32 copy of the new values."""
    A0 = M.diffusion3d_grf(N=40).A
    A1 = M.diffusion3d_grf(seed=77, N=40).A  # same pattern, other coefficients
    assert np.array_equal(A0.col_idx, A1.col_idx)
    b = np.random.default_rng(3).uniform(-1, 1, A0.n)
    s = solver(A0, {"precision": "MIXED", "outer_product": 1, "layout": "SLICED_ELL"})
    assert s.plan(0, "krylov")["df"]
    s.resetup(dev(A1.values))
    x, info = s.solve(dev(b))
    assert info.status == 0 and info.rel_res_true <= 1e-8
    xt, _ = O.Hierarchy(A1, {"rtol": 1e-13}).solve(b)
    assert np.linalg.norm(x.cpu().numpy() - xt) <= 1e-7 * np.linalg.norm(xt)
    s.close()
