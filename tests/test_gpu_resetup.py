"""GPU parity of the numeric re-setup (amg_resetup): new values on the same
pattern, the hierarchy's structure kept and every value recomputed, against
the oracle's re-setup of the same hierarchy (integers and values bit-exact),
and the solves, adjoints, cache and autograd paths built on it."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg  # noqa: F401  (sp.linalg)
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M
from paper_2606_09001_b300 import _lib
from paper_2606_09001_b300.autograd import amg_solve

pytestmark = pytest.mark.gpu

DEV = "cuda"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_solver(A, cfg=None):
    return api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values), cfg)


def ocfg(cfg):
    c = dict(cfg or {})
    c.pop("precision", None)
    c.pop("layout", None)
    c.pop("fuse_coarse", None)
    if isinstance(c.get("solver"), str):
        c["solver"] = _lib.SOLVERS[c["solver"]]
    return c


def same_hierarchy(s, h):
    assert s.info().nlevels == h.nlevels
    for l in range(h.nlevels):
        lv = h.level(l)
        rp, ci, v, _ = s.level(l, "A")
        assert np.array_equal(rp, lv.A.row_ptr) and np.array_equal(ci, lv.A.col_idx), f"A{l} pattern"
        assert np.array_equal(v.view(np.int64), lv.A.values.view(np.int64)), f"A{l} values"
        if l < h.nlevels - 1:
            assert np.array_equal(s.aggregates(l), lv.agg), f"aggregates {l}"
            for which, ref in (("P", lv.P), ("R", lv.R)):
                rp, ci, v, _ = s.level(l, which)
                assert np.array_equal(ci, ref.col_idx), f"{which}{l} pattern"
                assert np.array_equal(v.view(np.int64), ref.values.view(np.int64)), f"{which}{l} values"


def pairs():
    """(name, A0, A1, cfg): two matrices with one pattern and different values."""
    g = M.diffusion3d_grf
    return {
        "logk2d_40": (M.diffusion2d_logk(N=40).A, M.diffusion2d_logk(seed=77, N=40).A, {}),
        "grf3d_20": (g(N=20).A, g(seed=5, N=20).A, {}),
        "grf3d_33_stream": (g(N=33).A, g(seed=9, N=33).A, {}),
        "grf3d_33_mixed": (g(N=33).A, g(seed=9, N=33).A, {"precision": "MIXED"}),
        "poisson2d_64_tail": (M.poisson2d(64), M.diffusion_fv(np.exp(0.3 * np.random.default_rng(3).normal(size=(64, 64)))), {}),
    }


@pytest.mark.parametrize("name", list(pairs()))
def test_resetup_hierarchy_and_solve_match_oracle(name):
    A0, A1, cfg = pairs()[name]
    assert np.array_equal(A0.col_idx, A1.col_idx) and np.array_equal(A0.row_ptr, A1.row_ptr)
    s = gpu_solver(A0, cfg)
    s.resetup(dev(A1.values))
    h = O.Hierarchy(A0, ocfg(cfg)).resetup(A1.values)
    same_hierarchy(s, h)
    b = np.random.default_rng(4).uniform(-1, 1, A1.n)
    x, info = s.solve(dev(b))
    xo, io = h.solve(b)
    x = x.cpu().numpy()
    assert info.status == 0 and info.rel_res_true <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    tight = O.Hierarchy(A1, {"rtol": 1e-13})
    xt, _ = tight.solve(b)
    assert np.linalg.norm(x - xt) <= 1e-7 * np.linalg.norm(xt)


def test_resetup_same_values_reproduces_solve_bitwise():
    A = M.diffusion3d_grf(N=33).A
    s = gpu_solver(A)
    b = dev(np.random.default_rng(2).uniform(-1, 1, A.n))
    x1, i1 = s.solve(b)
    s.resetup(dev(A.values))
    x2, i2 = s.solve(b)
    assert torch.equal(x1, x2) and i1.iters == i2.iters


def test_resetup_host_values_and_cache_path():
    A0, A1, _ = pairs()["logk2d_40"]
    cache = api.SetupCache()
    rp, ci = dev(A0.row_ptr), dev(A0.col_idx)
    s0 = cache.get(rp, ci, dev(A0.values), api.make_config())
    s1 = cache.get(rp, ci, dev(A1.values), api.make_config())
    assert s1 is s0 and cache.resetups == 1 and s1.generation == 1
    direct = gpu_solver(A0)
    direct.resetup(A1.values)  # host values
    b = dev(np.random.default_rng(6).uniform(-1, 1, A1.n))
    xa, _ = s1.solve(b)
    xb, _ = direct.solve(b)
    assert torch.equal(xa, xb)


def test_resetup_nonsymmetric_adjoint_follows():
    """The cached hierarchy of A^T is re-set up with the transpose of the new values."""
    A0 = M.convection_diffusion_upwind(14)
    rng = np.random.default_rng(12)
    A1 = M.CSR(A0.row_ptr, A0.col_idx, A0.values * rng.uniform(0.8, 1.25, A0.nnz))
    cfg = {"solver": "BICGSTAB"}
    s = gpu_solver(A0, cfg)
    b = dev(rng.uniform(-1, 1, A0.n))
    g = rng.uniform(-1, 1, A0.n)
    x0, _ = s.solve(b)
    s.adjoint(x0, dev(g))  # builds the A^T hierarchy
    s.resetup(dev(A1.values))
    x, info = s.solve(b)
    lam, dA, ainfo = s.adjoint(x, dev(g))
    assert info.status == 0 and ainfo.status == 0 and ainfo.rel_res_true <= 1e-8
    A1s = sp.csr_matrix((A1.values, A1.col_idx, A1.row_ptr), shape=(A1.n, A1.n))
    lam_ref = np.linalg.solve(A1s.T.toarray(), g)
    lam = lam.cpu().numpy()
    assert np.linalg.norm(lam - lam_ref) <= 1e-6 * np.linalg.norm(lam_ref)


def test_resetup_errors():
    A = M.poisson2d(30)
    s = gpu_solver(A)
    # a nonsymmetric set of values on the symmetric pattern
    v = A.values.copy()
    v[1] *= 1.5
    with pytest.raises(api.AMGError) as e:
        s.resetup(dev(v))
    assert e.value.code == _lib.AMG_ERR_ARG
    s = gpu_solver(A, {"symmetric": 1})
    v = A.values.copy()
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    v[(rows == 5) & (A.col_idx == 5)] = 0.0
    with pytest.raises(api.AMGError) as e:
        s.resetup(dev(v))
    assert e.value.code == _lib.AMG_ERR_ZERO_DIAG
    blocks = [M.poisson2d(10), M.poisson2d(12)]
    Ab, off = M.block_diag(blocks)
    bs = api.BatchedSolver(dev(off), dev(Ab.row_ptr), dev(Ab.col_idx), dev(Ab.values))
    L = _lib.load()
    assert L.amg_resetup(bs._h, dev(Ab.values).data_ptr(), 0) == _lib.AMG_ERR_UNSUPPORTED


def test_autograd_interleaved_forwards_use_their_own_values():
    """Two forward solves with different values on one cached pattern, then the
    backward of the first: its gradient is that of the first values."""
    A0, A1, _ = pairs()["logk2d_40"]
    cache = api.SetupCache()
    rp, ci = dev(A0.row_ptr), dev(A0.col_idx)
    b = dev(np.random.default_rng(8).uniform(-1, 1, A0.n))
    v0 = dev(A0.values).requires_grad_(True)
    v1 = dev(A1.values).requires_grad_(True)
    x0 = amg_solve(rp, ci, v0, b, cache=cache)
    x1 = amg_solve(rp, ci, v1, b, cache=cache)
    (x0 ** 2).sum().backward()
    g_interleaved = v0.grad.clone()
    v0b = dev(A0.values).requires_grad_(True)
    xb = amg_solve(rp, ci, v0b, b, cache=api.SetupCache())
    (xb ** 2).sum().backward()
    assert torch.linalg.norm(g_interleaved - v0b.grad) <= 1e-6 * torch.linalg.norm(v0b.grad)
    del x1


@pytest.mark.parametrize("solver", ["CG", "BICGSTAB_NOPREC"])
def test_unpreconditioned_handle_keeps_the_finest_level_only(solver):
    """An unpreconditioned solver's handle builds no coarse levels: one level,
    no V-cycle to export, and a re-setup that only takes the new values."""
    A0 = M.tridiagonal_matrix(5000, 4.0)
    A1 = M.tridiagonal_matrix(5000, 3.0)
    s = gpu_solver(A0, {"solver": solver})
    assert s.info().nlevels == 1
    L = _lib.load()
    r = dev(np.ones(A0.n))
    z = torch.empty_like(r)
    assert L.amg_vcycle(s._h, r.data_ptr(), z.data_ptr(), None) == _lib.AMG_ERR_UNSUPPORTED
    b = np.random.default_rng(5).uniform(-1, 1, A1.n)
    s.resetup(dev(A1.values))
    x, info = s.solve(dev(b))
    _, io = O.Hierarchy(A1, {"solver": _lib.SOLVERS[solver]}).solve(b)
    A1s = sp.csr_matrix((A1.values, A1.col_idx, A1.row_ptr), shape=(A1.n, A1.n))
    xt = sp.linalg.spsolve(A1s.tocsc(), b)
    assert info.status == 0 and info.rel_res_true <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    assert np.linalg.norm(x.cpu().numpy() - xt) <= 1e-7 * np.linalg.norm(xt)
    lam, dA, ainfo = s.adjoint(x, dev(np.ones(A1.n)))
    assert ainfo.status == 0 and ainfo.rel_res_true <= 1e-8
