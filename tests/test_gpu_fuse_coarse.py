"""GPU parity of the cooperative launch of the coarse levels
(amg_config.fuse_coarse): the run of coarse levels below the streaming
threshold, with the dense end of the V-cycle, as one whole-GPU launch with a
grid barrier between its passes.

On hierarchies whose levels all stay below 16384 rows no operator has a timed
plan, so the cooperative launch (fuse_coarse = 2, which takes it even where
the single-cluster tail would fit) must give the same bits as one launch per
pass (fuse_coarse = 0): V-cycle, PCG and BiCGStab solves, the adjoint, mixed
precision, classical hierarchies, a re-setup.  Slowly coarsening operators
(1D, 2D) supply the smoothed levels between 2048 and 16384 rows that such
small problems need.  On a tridiagonal of 59000 rows and the 128^3 diffusion
hierarchy the cooperative launch runs behind streamed levels; the result
matches the per-pass cycle bit for bit whenever the two handles' timed
trials chose the same plans, and to rounding always.  The default
(fuse_coarse = 1) never takes the cooperative launch."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M

pytestmark = pytest.mark.gpu

DEV = "cuda"


def convdiff1d(n, pe=0.5):
    """Upwind 1D convection-diffusion tridiag(-1-pe, 2+pe, -1) (nonsymmetric)."""
    i = np.arange(n)
    rows = np.repeat(i, 3)
    cols = (rows + np.tile([-1, 0, 1], n)).astype(np.int64)
    vals = np.tile([-1.0 - pe, 2.0 + pe, -1.0], n)
    keep = (cols >= 0) & (cols < n)
    rp = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows[keep], minlength=n), out=rp[1:])
    return M.CSR(rp, cols[keep].astype(np.int32), vals[keep])


# Every level below 16384 rows (no timed plan anywhere), one smoothed level
# between the finest and the dense end (two for the classical tridiagonal).
SMALL = {
    # 15000 -> 4148 -> dense 1138
    "tri_15000": lambda: M.tridiagonal_matrix(15000),
    # 16129 -> 2295 -> dense 197
    "poisson2d_127": lambda: M.poisson2d(127),
    # nonsymmetric: BiCGStab, the adjoint on a hierarchy of A^T
    "convdiff1d_15000": lambda: convdiff1d(15000),
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def solver(A, cfg):
    return api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values), cfg)


def launched(s, fn):
    """Names of the traced launches of fn()."""
    s.profile(True)
    fn()
    _, recs = s.profile_records()
    s.profile(False)
    return {r["name"] for r in recs if r["launches"] > 0}


def same_bits(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("name", list(SMALL))
def test_vcycle_bits_match_per_pass(name, precision):
    A = SMALL[name]()
    assert A.n < 16384
    r = np.random.default_rng(3).uniform(-1, 1, A.n)
    s0 = solver(A, {"precision": precision, "fuse_coarse": 0})
    s2 = solver(A, {"precision": precision, "fuse_coarse": 2})
    z0 = s0.vcycle(dev(r)).cpu().numpy()
    names = launched(s2, lambda: s2.vcycle(dev(r)))
    assert "mid" in names and "tail" not in names and "coarse" not in names, names
    assert "mid" not in launched(s0, lambda: s0.vcycle(dev(r)))
    z2 = s2.vcycle(dev(r)).cpu().numpy()
    assert same_bits(z0, z2)
    # and against the oracle
    zo = O.Hierarchy(A).vcycle(r)
    tol = 1e-12 if precision == "FP64" else 1e-5
    assert np.linalg.norm(z2 - zo) <= tol * np.linalg.norm(zo)


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("name", list(SMALL))
def test_solve_and_adjoint_bits_match_per_pass(name, precision):
    A = SMALL[name]()
    cfg = {"solver": "BICGSTAB"} if name.startswith("convdiff") else {}
    rng = np.random.default_rng(11)
    b, g = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    out = []
    for fuse in (0, 2):
        s = solver(A, dict(cfg, precision=precision, fuse_coarse=fuse))
        x, info = s.solve(dev(b))
        assert info.status == 0 and info.rel_res_true <= 1e-8
        lam, dA, ainfo = s.adjoint(x, dev(g))
        assert ainfo.status == 0
        out.append((x.cpu().numpy(), info.iters, lam.cpu().numpy(), dA.cpu().numpy(), ainfo.iters))
    (x0, i0, l0, d0, a0), (x2, i2, l2, d2, a2) = out
    assert i0 == i2 and a0 == a2
    assert same_bits(x0, x2) and same_bits(l0, l2) and same_bits(d0, d2)


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("case", ["adjoint_reuse", "classical_tri", "classical_grf"])
def test_adjoint_reuse_and_classical_bits_match_per_pass(case, precision):
    """Transposed-hierarchy reuse on the nonsymmetric operator; classical
    hierarchies with two smoothed levels in the cooperative launch
    (tridiagonal: 15000 -> 6489 -> 2825 -> dense 1221) and with one (24^3
    diffusion: 13824 -> 4474 -> dense 936)."""
    A, extra = {
        "adjoint_reuse": (lambda: SMALL["convdiff1d_15000"](), {"solver": "BICGSTAB", "adjoint_reuse": 1}),
        "classical_tri": (lambda: M.tridiagonal_matrix(15000), {"amg_type": "CLASSICAL"}),
        "classical_grf": (lambda: M.diffusion3d_grf(N=24).A, {"amg_type": "CLASSICAL"}),
    }[case]
    A = A()
    rng = np.random.default_rng(5)
    b, g = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    res = []
    for fuse in (0, 2):
        s = solver(A, dict(extra, precision=precision, fuse_coarse=fuse))
        if fuse == 2:
            assert "mid" in launched(s, lambda: s.vcycle(dev(b)))
        x, info = s.solve(dev(b))
        assert info.status == 0 and info.rel_res_true <= 1e-8
        lam, _, ainfo = s.adjoint(x, dev(g))
        assert ainfo.status == 0
        res.append((x.cpu().numpy(), lam.cpu().numpy(), info.iters, ainfo.iters))
    assert res[0][2:] == res[1][2:]
    assert same_bits(res[0][0], res[1][0]) and same_bits(res[0][1], res[1][1])


def test_resetup_bits_match_per_pass():
    A0 = M.tridiagonal_matrix(15000)
    A1 = M.tridiagonal_matrix(15000, 2.5, -1.1)
    b = np.random.default_rng(2).uniform(-1, 1, A0.n)
    xs = []
    for fuse in (0, 2):
        s = solver(A0, {"fuse_coarse": fuse})
        s.resetup(dev(A1.values))
        x, info = s.solve(dev(b))
        assert info.status == 0
        xs.append(x.cpu().numpy())
    assert same_bits(xs[0], xs[1])
    xo, _ = O.solve(A1, b, {"rtol": 1e-13})
    assert np.linalg.norm(xs[1] - xo) <= 1e-7 * np.linalg.norm(xo)


def test_two_level_hierarchy_keeps_the_per_pass_cycle():
    """With no smoothed level between the finest and the dense end there is
    nothing to fuse: fuse_coarse = 2 launches the per-pass cycle (24^3
    diffusion: 13824 -> dense 520)."""
    A = M.diffusion3d_grf(N=24).A
    r = np.random.default_rng(4).uniform(-1, 1, A.n)
    s0, s2 = solver(A, {"fuse_coarse": 0}), solver(A, {"fuse_coarse": 2})
    names = launched(s2, lambda: s2.vcycle(dev(r)))
    assert "mid" not in names and "coarse" in names, names
    assert same_bits(s0.vcycle(dev(r)).cpu().numpy(), s2.vcycle(dev(r)).cpu().numpy())


def test_default_takes_the_tail_or_the_per_pass_cycle():
    A = SMALL["tri_15000"]()
    r = np.random.default_rng(6).uniform(-1, 1, A.n)
    s = solver(A, {})
    names = launched(s, lambda: s.vcycle(dev(r)))
    assert "mid" not in names and "tail" in names, names


def test_fuse_coarse_is_validated():
    A = SMALL["poisson2d_127"]()
    for bad in (-1, 3):
        with pytest.raises(api.AMGError):
            solver(A, {"fuse_coarse": bad})


def plans(s):
    return [[s.plan(l, op) for op in ("pre", "post", "P", "R") + (("krylov",) if l == 0 else ())]
            for l in range(s.info().nlevels)]


CASES_STREAMED = {
    # 59000 (streamed) -> 16265 -> 4493 -> dense 1233: two smoothed levels in
    # the cooperative launch behind a streamed finest level
    "tri_59000": lambda: M.tridiagonal_matrix(59000),
    # 128^3 diffusion: 2097152 -> 188816 (streamed) -> 12042 -> dense 1137,
    # a level whose operator holds more entries than the single-cluster tail
    # takes
    "grf3d_128": lambda: M.diffusion3d_grf(N=128).A,
}


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("name", list(CASES_STREAMED))
def test_streamed_hierarchies_run_the_cooperative_launch(name, precision):
    """The streamed operators' plans come from a timed trial per handle:
    where both handles chose the same plans the cycles agree bit for bit,
    else to rounding."""
    A = CASES_STREAMED[name]()
    rng = np.random.default_rng(9)
    r = rng.uniform(-1, 1, A.n)
    s1 = solver(A, {"precision": precision, "fuse_coarse": 2})
    names = launched(s1, lambda: s1.vcycle(dev(r)))
    assert "mid" in names and "tail" not in names, names
    z1 = s1.vcycle(dev(r)).cpu().numpy()
    s0 = solver(A, {"precision": precision, "fuse_coarse": 0})
    z0 = s0.vcycle(dev(r)).cpu().numpy()
    if plans(s0) == plans(s1):
        assert same_bits(z0, z1)
    tol = 1e-12 if precision == "FP64" else 1e-5
    assert np.linalg.norm(z1 - z0) <= tol * np.linalg.norm(z0)
    if A.n < 100000:
        zo = O.Hierarchy(A).vcycle(r)
        assert np.linalg.norm(z1 - zo) <= tol * np.linalg.norm(zo)
    b = rng.uniform(-1, 1, A.n)
    x, info = s1.solve(dev(b))
    assert info.status == 0 and info.rel_res_true <= 1e-8
    x0, info0 = s0.solve(dev(b))
    assert abs(info.iters - info0.iters) <= 1
    xn, x0n = x.cpu().numpy(), x0.cpu().numpy()
    assert np.linalg.norm(xn - x0n) <= 1e-6 * np.linalg.norm(x0n)
