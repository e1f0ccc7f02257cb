"""GPU parity of the batched solve (many independent systems, up to 8
right-hand sides each) against the FP64 CPU oracle run on every system
alone: the batch's hierarchy must hold, for every system, exactly the
oracle's hierarchy of that system (integers and values bit-exact), and every
(system, right-hand side) pair must converge like the oracle's solve of
that pair."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle as O
from paper_2606_09001_b300 import api, matrices as M
from paper_2606_09001_b300 import _lib

pytestmark = pytest.mark.gpu

DEV = "cuda"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def small_batch():
    """Systems of mixed kinds and sizes: one ends on level 0 (64 rows), one
    after a single coarsening, several go three or more levels deep."""
    blocks = [
        M.poisson2d(23),
        M.poisson2d(8),                      # 64 rows: solved densely on level 0
        M.diffusion3d_grf(N=10).A,
        M.tridiagonal_matrix(300, 2.5),
        M.poisson2d(40),
        M.poisson3d(9),
        M.poisson2d(12),
        M.diffusion2d_logk(N=30).A,
    ]
    A, off = M.block_diag(blocks)
    return blocks, A, off


def batched_solver(A, off, cfg=None):
    return api.BatchedSolver(dev(off), dev(A.row_ptr), dev(A.col_idx), dev(A.values), cfg)


def csr_block(rp, ci, v, r0, r1, c0):
    """Rows r0..r1-1 of a CSR as a CSR of their own, columns shifted by -c0."""
    a, b = rp[r0], rp[r1]
    return rp[r0:r1 + 1] - a, ci[a:b] - c0, v[a:b]


def check_hierarchy(blocks, s, cfg=None):
    hs = [O.Hierarchy(B, cfg or {}) for B in blocks]
    L = s.info().nlevels
    assert L == max(h.nlevels for h in hs)
    for l in range(L):
        sys_ids, off, fin = s.batch_level(l)
        want = [k for k, h in enumerate(hs) if h.nlevels > l]
        assert list(sys_ids) == want, f"systems on level {l}"
        rpA, ciA, vA, _ = s.level(l, "A")
        if l < L - 1:
            nsys_next, off_next, _ = s.batch_level(l + 1)
            next_pos = {int(k): j for j, k in enumerate(nsys_next)}
            agg = s.aggregates(l)
            rpP, ciP, vP, _ = s.level(l, "P")
            rpR, ciR, vR, _ = s.level(l, "R")
        for j, k in enumerate(sys_ids):
            h = hs[k]
            lv = h.level(l)
            r0, r1 = off[j], off[j + 1]
            assert r1 - r0 == lv.A.n, f"rows of system {k} on level {l}"
            assert fin[j] == (h.nlevels == l + 1), f"final flag of system {k} on level {l}"
            rp, ci, v = csr_block(rpA, ciA, vA, r0, r1, r0)
            assert np.array_equal(rp, lv.A.row_ptr) and np.array_equal(ci, lv.A.col_idx), f"A{l} pattern, system {k}"
            assert np.array_equal(v.view(np.int64), lv.A.values.view(np.int64)), f"A{l} values, system {k}"
            if fin[j]:
                if l < L - 1:
                    assert np.all(agg[r0:r1] < 0), "rows of a finished system are not aggregated"
                    assert np.all(np.diff(rpP[r0:r1 + 1]) == 0), "P rows of a finished system are empty"
                continue
            c0 = off_next[next_pos[int(k)]]
            assert np.array_equal(agg[r0:r1] - c0, lv.agg), f"aggregates level {l}, system {k}"
            rp, ci, v = csr_block(rpP, ciP, vP, r0, r1, c0)
            assert np.array_equal(rp, lv.P.row_ptr) and np.array_equal(ci, lv.P.col_idx), f"P{l} pattern, system {k}"
            assert np.array_equal(v.view(np.int64), lv.P.values.view(np.int64)), f"P{l} values, system {k}"
            nc = lv.R.n
            rp, ci, v = csr_block(rpR, ciR, vR, c0, c0 + nc, r0)
            assert np.array_equal(rp, lv.R.row_ptr) and np.array_equal(ci, lv.R.col_idx), f"R{l} pattern, system {k}"
            assert np.array_equal(v.view(np.int64), lv.R.values.view(np.int64)), f"R{l} values, system {k}"
    return hs


@pytest.mark.parametrize("prec", ["FP64", "MIXED"])
def test_batched_hierarchy_matches_each_system(prec):
    blocks, A, off = small_batch()
    s = batched_solver(A, off, {"precision": prec})
    check_hierarchy(blocks, s)


def test_batched_hierarchy_small_coarse_l1():
    blocks, A, off = small_batch()
    cfg = {"smoother": "L1_JACOBI", "coarse_max": 16}
    s = batched_solver(A, off, cfg)
    check_hierarchy(blocks, s, {"smoother": _lib.SMOOTHERS["L1_JACOBI"], "coarse_max": 16})


@pytest.mark.parametrize("prec,nrhs", [("FP64", 8), ("FP64", 3), ("MIXED", 8)])
def test_batched_solve_parity(prec, nrhs):
    blocks, A, off = small_batch()
    B = np.random.default_rng(11).uniform(-1, 1, (A.n, nrhs))
    s = batched_solver(A, off, {"precision": prec})
    X, its, rel, info = s.solve(dev(B))
    X = X.cpu().numpy()
    assert info.status == 0, _lib.status_string(info.status)
    assert its.shape == (len(blocks), nrhs) and rel.shape == (len(blocks), nrhs)
    assert np.all(rel <= 1e-8)
    for k, Bk in enumerate(blocks):
        r0, r1 = off[k], off[k + 1]
        h = O.Hierarchy(Bk)
        ht = O.Hierarchy(Bk, {"rtol": 1e-13})
        for r in range(nrhs):
            b = np.ascontiguousarray(B[r0:r1, r])
            xo, io = h.solve(b)
            xt, _ = ht.solve(b)
            x = X[r0:r1, r]
            assert abs(int(its[k, r]) - io.iters) <= 2, (k, r, its[k, r], io.iters)
            if prec == "FP64":
                # same algorithm, same hierarchy: the iterates agree to rounding
                assert np.linalg.norm(x - xo) <= 1e-7 * np.linalg.norm(xo), (k, r)
            assert np.linalg.norm(x - xt) <= 1e-7 * np.linalg.norm(xt), (k, r)
            Ak = sp.csr_matrix((Bk.values, Bk.col_idx, Bk.row_ptr), shape=(Bk.n, Bk.n))
            assert np.linalg.norm(Ak @ x - b) <= 1.0001e-8 * np.linalg.norm(b), (k, r)


def test_batched_zero_columns_and_host_arrays():
    blocks, A, off = small_batch()
    B = np.random.default_rng(4).uniform(-1, 1, (A.n, 5))
    B[off[2]:off[3], 1] = 0.0          # one system's right-hand side is zero
    B[:, 4] = 0.0                      # a whole column is zero
    s = batched_solver(A, off)
    X, its, rel, info = s.solve(B)     # host in, host out
    assert isinstance(X, np.ndarray)
    assert info.status == 0
    assert np.all(X[off[2]:off[3], 1] == 0.0) and its[2, 1] == 0 and rel[2, 1] == 0.0
    assert np.all(X[:, 4] == 0.0) and np.all(its[:, 4] == 0)
    Xd, its_d, _, _ = s.solve(dev(B))
    assert np.array_equal(X, Xd.cpu().numpy()) and np.array_equal(its, its_d)


def test_batched_deterministic_and_reusable():
    blocks, A, off = small_batch()
    s = batched_solver(A, off)
    B1 = np.random.default_rng(1).uniform(-1, 1, (A.n, 8))
    B2 = np.random.default_rng(2).uniform(-1, 1, (A.n, 8))
    X1, i1, _, _ = s.solve(dev(B1))
    X2, _, _, _ = s.solve(dev(B2))
    X1b, i1b, _, _ = s.solve(dev(B1))
    assert torch.equal(X1, X1b) and np.array_equal(i1, i1b)
    assert not torch.equal(X1, X2)


def test_batched_single_system_matches_plain_solver():
    A = M.poisson2d(45)
    off = np.array([0, A.n], np.int32)
    b = np.random.default_rng(8).uniform(-1, 1, A.n)
    s = batched_solver(A, off)
    X, its, rel, info = s.solve(dev(b.reshape(-1, 1)))
    x1, i1 = api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values)).solve(dev(b))
    assert abs(int(its[0, 0]) - i1.iters) <= 1
    assert torch.linalg.norm(X[:, 0] - x1) <= 1e-9 * torch.linalg.norm(x1)


def test_batched_errors():
    blocks, A, off = small_batch()
    s = batched_solver(A, off)
    with pytest.raises(api.AMGError) as e:
        s.solve(dev(np.zeros((A.n, 9))))
    assert e.value.code == _lib.AMG_ERR_ARG
    L = _lib.load()
    x = dev(np.zeros(A.n))
    assert L.amg_solve(s._h, x.data_ptr(), x.data_ptr(), 0, None) == _lib.AMG_ERR_ARG
    with pytest.raises(api.AMGError) as e:
        batched_solver(A, off, {"solver": "BICGSTAB"})
    assert e.value.code == _lib.AMG_ERR_UNSUPPORTED
    # a row of system 0 coupling into system 1
    rp, ci, v = A.row_ptr.copy(), A.col_idx.copy(), A.values.copy()
    last = rp[off[1]] - 1                  # last entry of system 0's last row
    ci[last] = off[1]                      # still ascending: first column of system 1
    with pytest.raises(api.AMGError) as e:
        api.BatchedSolver(dev(off), dev(rp), dev(ci), dev(v))
    assert e.value.code == _lib.AMG_ERR_BAD_CSR
    bad_off = off.copy()
    bad_off[-1] -= 1
    with pytest.raises(api.AMGError) as e:
        batched_solver(A, bad_off)
    assert e.value.code == _lib.AMG_ERR_ARG


@pytest.mark.slow
def test_batched_full_size_sampled():
    """The batched Poisson workload at full size (256 systems, 8 right-hand
    sides) in the configuration the benchmark times: every pair converges,
    and sampled systems match the oracle run on them alone."""
    w = M.batched_poisson2d()
    off = w.extra["sys_off"]
    s = batched_solver(w.A, off, {"precision": "MIXED"})
    X, its, rel, info = s.solve(dev(w.b))
    assert info.status == 0 and np.all(rel <= 1e-8)
    X = X.cpu().numpy()
    sides = w.extra["sides"]
    for k in (int(np.argmin(sides)), 0, int(np.argmax(sides))):
        Bk = M.poisson2d(int(sides[k]))
        r0, r1 = off[k], off[k + 1]
        ht = O.Hierarchy(Bk, {"rtol": 1e-13})
        _, io = O.Hierarchy(Bk).solve(np.ascontiguousarray(w.b[r0:r1, 0]))
        for r in (0, 7):
            b = np.ascontiguousarray(w.b[r0:r1, r])
            xt, _ = ht.solve(b)
            assert np.linalg.norm(X[r0:r1, r] - xt) <= 1e-7 * np.linalg.norm(xt), (k, r)
        assert abs(int(its[k, 0]) - io.iters) <= 2
