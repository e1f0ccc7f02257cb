"""Pins for the FP64 CPU oracle: every check compares it with something other
than itself -- closed-form eigenpairs, dense direct solves and products done
by numpy/scipy, brute-force graph enumeration, finite differences and the
paper's worked examples (Sec. 3.1, 3.2).  CPU only."""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle as O
from paper_2606_09001_b300 import matrices as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")


def to_sp(A):
    return sp.csr_matrix((A.values, A.col_idx, A.row_ptr), shape=(A.n, A.n))


def lvl_sp(m, ncols):
    return sp.csr_matrix((m.values, m.col_idx, m.row_ptr), shape=(m.n, ncols))


# --------------------------------------------------------------------------
# SpMV against closed-form eigenpairs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,d", [(50, 2.0), (33, 4.0)])
def test_spmv_1d_eigenpairs(n, d):
    A = M.tridiagonal_matrix(n, d)
    for k in (1, 7, n):
        v = np.sin(k * np.pi * np.arange(1, n + 1) / (n + 1))
        lam = d - 2.0 * np.cos(k * np.pi / (n + 1))
        assert np.linalg.norm(O.spmv(A, v) - lam * v) <= 1e-13 * np.linalg.norm(v)


def test_spmv_2d_eigenpairs():
    s = 24
    A = M.poisson2d(s)
    t = np.arange(1, s + 1)
    for j, k in [(1, 1), (3, 5), (24, 2)]:
        v = np.outer(np.sin(k * np.pi * t / (s + 1)), np.sin(j * np.pi * t / (s + 1))).reshape(-1)
        lam = 4 - 2 * np.cos(j * np.pi / (s + 1)) - 2 * np.cos(k * np.pi / (s + 1))
        assert np.linalg.norm(O.spmv(A, v) - lam * v) <= 1e-13 * np.linalg.norm(v)


def test_transpose_matches_scipy():
    rng = np.random.default_rng(0)
    S = sp.random(40, 27, density=0.2, random_state=1, format="csr")
    S.sort_indices()
    rp, ci, v = O.transpose(S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data, 27)
    T = S.T.tocsr()
    T.sort_indices()
    assert np.array_equal(rp, T.indptr) and np.array_equal(ci, T.indices)
    assert np.array_equal(v, T.data)
    del rng


# --------------------------------------------------------------------------
# Validation
# --------------------------------------------------------------------------

def test_validate_codes():
    A = M.poisson2d(4)
    assert O.validate(A) == O.OK
    bad = M.CSR(A.row_ptr.copy(), A.col_idx.copy(), A.values.copy())
    bad.col_idx[1], bad.col_idx[0] = bad.col_idx[0], bad.col_idx[1]
    assert O.validate(bad) == O.ERR_BAD_CSR
    bad = M.CSR(A.row_ptr.copy(), A.col_idx.copy(), A.values.copy())
    bad.col_idx[-1] = A.n
    assert O.validate(bad) == O.ERR_BAD_CSR
    bad = M.CSR(A.row_ptr.copy(), A.col_idx.copy(), A.values.copy())
    bad.values[0] = 0.0  # row 0 stores its diagonal first
    assert O.validate(bad) == O.ERR_ZERO_DIAG
    bad = M.CSR(A.row_ptr.copy(), A.col_idx.copy(), A.values.copy())
    bad.row_ptr[2] = bad.row_ptr[1] - 1
    assert O.validate(bad) == O.ERR_BAD_CSR


# --------------------------------------------------------------------------
# Strength of connection
# --------------------------------------------------------------------------

def test_strength_poisson_all_links_strong():
    A = M.poisson2d(9)
    srp, sci = O.strength(A, 0.08)
    D = A.to_dense()
    off = (D != 0) & ~np.eye(A.n, dtype=bool)
    S = np.zeros_like(off)
    S[np.repeat(np.arange(A.n), np.diff(srp)), sci] = True
    assert np.array_equal(S, off)


def test_strength_anisotropic_keeps_strong_direction():
    # -u_xx - eps u_yy with eps = 1e-3: y-links |a| = eps fail the test
    # (eps^2 < 0.08^2 (2+2eps)^2), x-links pass -> S is the union of x-lines.
    s, eps = 8, 1e-3
    n = s * s
    D = np.zeros((n, n))
    for i in range(n):
        x, y = i % s, i // s
        D[i, i] = 2 + 2 * eps
        if x > 0: D[i, i - 1] = -1
        if x < s - 1: D[i, i + 1] = -1
        if y > 0: D[i, i - s] = -eps
        if y < s - 1: D[i, i + s] = -eps
    A = M.CSR(*_dense_to_csr(D))
    srp, sci = O.strength(A, 0.08)
    rows = np.repeat(np.arange(n), np.diff(srp))
    assert np.all(np.abs(rows - sci) == 1) and np.all(rows // s == sci // s)
    assert sci.size == 2 * s * (s - 1)


def test_strength_threshold_equality_is_strong_and_union_symmetric():
    # theta = 0.5: a_01^2 = 1 = 0.25 * |2 * 2| -> strong by equality.
    D = np.array([[2.0, -1.0, 0.0], [-1.0, 2.0, -0.1], [0.0, -3.0, 4.0]])
    A = M.CSR(*_dense_to_csr(D))
    srp, sci = O.strength(A, 0.5)
    S = {(i, j) for i in range(3) for j in sci[srp[i]:srp[i + 1]]}
    # (1,2): 0.01 < 0.25*8 weak; (2,1): 9 >= 0.25*8 strong -> union keeps both
    assert S == {(0, 1), (1, 0), (1, 2), (2, 1)}


def _dense_to_csr(D):
    Ssp = sp.csr_matrix(D)
    Ssp.sort_indices()
    # keep explicit diagonal even when zero is impossible here
    return Ssp.indptr.astype(np.int32), Ssp.indices.astype(np.int32), Ssp.data.astype(np.float64)


# --------------------------------------------------------------------------
# MIS-2 and aggregation
# --------------------------------------------------------------------------

def _dist2_sets(srp, sci):
    import networkx as nx
    n = srp.shape[0] - 1
    G = nx.Graph()
    G.add_nodes_from(range(n))
    for i in range(n):
        for j in sci[srp[i]:srp[i + 1]]:
            G.add_edge(i, int(j))
    return G, {i: set(nx.single_source_shortest_path_length(G, i, cutoff=2)) for i in range(n)}


def _check_mis2(srp, sci, root):
    _, ball = _dist2_sets(srp, sci)
    R = np.flatnonzero(root)
    for i in R:  # independence: no other root within distance 2
        assert not (ball[i] - {i}) & set(R.tolist())
    for i in range(len(root)):  # maximality: every node within distance 2 of a root
        assert ball[i] & set(R.tolist())


def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    U = np.triu(rng.random((n, n)) < p, 1)
    Adj = U | U.T
    srp = np.zeros(n + 1, np.int32)
    srp[1:] = np.cumsum(Adj.sum(1))
    sci = np.concatenate([np.flatnonzero(Adj[i]) for i in range(n)]).astype(np.int32) if Adj.any() else np.zeros(0, np.int32)
    return srp, sci


def test_fmix32_is_murmur3_finaliser_and_bijective():
    # Appleby's MurmurHash3 fmix32: xor-shift 16, * 0x85ebca6b, xor-shift 13,
    # * 0xc2b2ae35, xor-shift 16 (mod 2^32).
    def ref(h):
        h ^= h >> 16; h = (h * 0x85EBCA6B) & 0xFFFFFFFF
        h ^= h >> 13; h = (h * 0xC2B2AE35) & 0xFFFFFFFF
        return h ^ (h >> 16)
    for v in (0, 1, 2, 12345, 2**31 - 1, 2**32 - 1):
        assert O.fmix32(v) == ref(v)
    vals = {O.fmix32(i) for i in range(20000)}
    assert len(vals) == 20000 and O.fmix32(0) == 0


@pytest.mark.parametrize("seed", range(6))
def test_mis2_tiny_graphs_lexicographically_first(seed):
    n = 10 + seed % 3
    srp, sci = _random_graph(n, 0.25, seed)
    root, _ = O.mis2(srp, sci, "greedy")
    root_r, _ = O.mis2(srp, sci, "rounds")
    assert np.array_equal(root, root_r)
    _, ball = _dist2_sets(srp, sci)
    # enumerate every distance-2 independent, maximal set; the greedy set is
    # the one that is lexicographically first in decreasing-priority order
    order = sorted(range(n), key=lambda i: (O.fmix32(i), i), reverse=True)
    best = None
    for mask in range(1 << n):
        R = [i for i in range(n) if mask >> i & 1]
        if any((ball[i] - {i}) & set(R) for i in R):
            continue
        if not all(ball[i] & set(R) for i in range(n)):
            continue
        key = tuple(1 if (mask >> i & 1) else 0 for i in order)
        if best is None or key > best[0]:
            best = (key, R)
    assert sorted(np.flatnonzero(root).tolist()) == sorted(best[1])


@pytest.mark.parametrize("maker", [lambda: M.poisson2d(20), lambda: M.poisson3d(7),
                                   lambda: M.convection_diffusion_upwind(6)])
def test_mis2_grid_independent_maximal_and_rounds_equal(maker):
    A = maker()
    srp, sci = O.strength(A, 0.08)
    root, _ = O.mis2(srp, sci, "greedy")
    root_r, nr = O.mis2(srp, sci, "rounds")
    assert np.array_equal(root, root_r) and nr < 40
    _check_mis2(srp, sci, root)


def test_mis2_rounds_equal_greedy_random_graphs():
    for seed in range(5):
        srp, sci = _random_graph(300, 0.01 + 0.01 * seed, seed + 10)
        a, _ = O.mis2(srp, sci, "greedy")
        b, _ = O.mis2(srp, sci, "rounds")
        assert np.array_equal(a, b)
        _check_mis2(srp, sci, a)


@pytest.mark.parametrize("maker", [lambda: M.poisson2d(17), lambda: M.poisson3d(6),
                                   lambda: M.convection_diffusion_upwind(6),
                                   lambda: M.diffusion_fv(np.exp(np.random.default_rng(3).normal(size=(12, 12))))])
def test_aggregates_partition_and_connected(maker):
    import networkx as nx
    A = maker()
    srp, sci = O.strength(A, 0.08)
    root, _ = O.mis2(srp, sci)
    agg, nc = O.aggregate(A, srp, sci, root.astype(np.int32))
    assert agg.min() == 0 and agg.max() == nc - 1
    R = np.flatnonzero(root)
    assert nc == R.size and np.array_equal(agg[R], np.arange(nc))  # ids by node index
    G, ball = _dist2_sets(srp, sci)
    for J in range(nc):
        members = np.flatnonzero(agg == J)
        assert nx.is_connected(G.subgraph(members.tolist()))
        assert set(members.tolist()) <= ball[R[J]]  # radius 2 around its root


def _strength_by_definition(A_sp, theta):
    """S by its definition, written with scipy: j is strong for i (i != j)
    when a_ij^2 >= theta^2 |a_ii a_jj|, and S is that relation united with
    its transpose.  Returns a set of (i, j)."""
    Acoo = A_sp.tocoo()
    d = A_sp.diagonal()
    off = Acoo.row != Acoo.col
    r, c, v = Acoo.row[off], Acoo.col[off], Acoo.data[off]
    strong = v * v >= (theta * theta) * np.abs(d[r] * d[c])
    pairs = set(zip(r[strong].tolist(), c[strong].tolist()))
    return pairs | {(j, i) for (i, j) in pairs}


def _pairs(srp, sci):
    rows = np.repeat(np.arange(srp.shape[0] - 1), np.diff(srp))
    return set(zip(rows.tolist(), sci.tolist()))


def test_strength_threshold_halves_per_level():
    """Every level's strength graph is the definition evaluated on that
    level's operator with theta_l = 0.08 * 2^-l (reading: the threshold halves
    per level), and the level's aggregates are the MIS-2 aggregation of that
    graph.  On a 3D GRF hierarchy a constant threshold gives other graphs on
    the coarse levels, so dropping or doubling the halving fails here."""
    A = M.diffusion3d_grf(N=20).A
    h = O.Hierarchy(A, {"coarse_max": 8})
    assert h.nlevels >= 4
    differs = 0
    for l in range(min(4, h.nlevels - 1)):
        lv = h.level(l)
        Al = lvl_sp(lv.A, lv.A.n)
        srp, sci = h.strength(l)
        got = _pairs(srp, sci)
        assert got == _strength_by_definition(Al, 0.08 * 2.0 ** -l), f"level {l}"
        if l > 0:
            differs += got != _strength_by_definition(Al, 0.08)
            differs += got != _strength_by_definition(Al, 0.08 * 2.0 ** -(l + 1))
        root, _ = O.mis2(srp, sci)
        agg, nc = O.aggregate(lv.A, srp, sci, root.astype(np.int32))
        assert np.array_equal(agg, lv.agg) and nc == h.level(l + 1).A.n, f"level {l}"
    assert differs >= 2  # the case tells the per-level threshold from its neighbours


def _check_phase3(A, srp, sci, root, agg):
    """Aggregation phases 2-3 by brute force: roots are numbered by index; a
    non-root adjacent to a root joins it (the root is unique); every other
    node joins the aggregate of its strong neighbour assigned in phase 2 with
    the largest |a_ij| (0 when (i, j) is not stored), smallest j on ties.
    Returns how many phase-3 nodes that rule decides differently from
    'the first assigned neighbour'."""
    n = A.n
    R = np.flatnonzero(root)
    assert np.array_equal(agg[R], np.arange(R.size))
    absA = {}
    for i in range(n):
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            absA[(i, int(A.col_idx[k]))] = abs(A.values[k])
    snap = np.full(n, -1)
    snap[R] = np.arange(R.size)
    for i in range(n):
        if root[i]:
            continue
        nb = [int(j) for j in sci[srp[i]:srp[i + 1]] if root[j]]
        assert len(nb) <= 1  # independence: at most one adjacent root
        if nb:
            snap[i] = snap[nb[0]]
            assert agg[i] == snap[i]
    telling = 0
    for i in range(n):
        if snap[i] >= 0:
            continue
        cand = [int(j) for j in sci[srp[i]:srp[i + 1]] if snap[j] >= 0]
        assert cand, "maximality leaves every node a phase-2 neighbour"
        best = min(cand, key=lambda j: (-absA.get((i, j), 0.0), j))
        assert agg[i] == snap[best], (i, cand, best)
        telling += snap[cand[0]] != snap[best]
    return telling


@pytest.mark.parametrize("maker", [
    lambda: M.diffusion_fv(np.exp(np.random.default_rng(17).normal(size=(30, 30)))),
    lambda: M.diffusion_fv(np.exp(np.random.default_rng(18).normal(size=(9, 9, 9)))),
])
def test_aggregation_phase3_joins_largest_coupling(maker):
    A = maker()
    srp, sci = O.strength(A, 0.08)
    root, _ = O.mis2(srp, sci)
    agg, _ = O.aggregate(A, srp, sci, root.astype(np.int32))
    assert _check_phase3(A, srp, sci, root, agg) > 0


def test_aggregation_phase3_on_a_coarse_level():
    """The same brute-force rule on the level-1 operator of a 3D GRF
    hierarchy (distinct Galerkin couplings), with the level's own graph."""
    h = O.Hierarchy(M.diffusion3d_grf(N=20).A, {"coarse_max": 8})
    lv = h.level(1)
    srp, sci = h.strength(1)
    root, _ = O.mis2(srp, sci)
    assert _check_phase3(lv.A, srp, sci, root, lv.agg) > 0


# --------------------------------------------------------------------------
# Prolongator, Galerkin, hierarchy
# --------------------------------------------------------------------------

def test_gershgorin_rho_poisson_closed_form():
    s = 64
    h = O.Hierarchy(M.poisson2d(s))
    rho = h.level(0).rho
    assert rho == 2.0  # interior rows: (4 + 4) / 4
    assert 1 + np.cos(np.pi / (s + 1)) <= rho  # true rho(D^-1 A)


@pytest.mark.parametrize("maker", [lambda: M.poisson2d(16), lambda: M.poisson3d(8),
                                   lambda: M.convection_diffusion_upwind(8),
                                   lambda: M.diffusion_fv(np.exp(np.random.default_rng(5).normal(size=(16, 16))))])
def test_prolongator_and_galerkin_against_dense(maker):
    A = maker()
    h = O.Hierarchy(A, {"coarse_max": 8})
    assert h.nlevels >= 2
    for l in range(h.nlevels - 1):
        lv, nx_ = h.level(l), h.level(l + 1)
        n, nc = lv.A.n, nx_.A.n
        Ad = lvl_sp(lv.A, n).toarray()
        T = np.zeros((n, nc))
        T[np.arange(n), lv.agg] = 1.0
        assert np.array_equal(T.sum(1), np.ones(n))
        d = np.diag(Ad)
        rho = np.max(np.abs(Ad).sum(1) / np.abs(d))
        assert lv.rho == pytest.approx(rho, rel=1e-15)
        Pd = (np.eye(n) - (4.0 / 3.0) / rho * (Ad / d[:, None])) @ T
        P = lvl_sp(lv.P, nc).toarray()
        assert np.allclose(P, Pd, rtol=0, atol=1e-14)
        # structural pattern: columns of P = aggregates touched by the row of A
        pat = (np.abs(Ad) > 0).astype(float) @ T > 0
        assert np.array_equal(lvl_sp(lv.P, nc).toarray() != 0, pat & (P != 0))
        assert np.array_equal(np.diff(lv.P.row_ptr), pat.sum(1))
        # P 1 = 1 on rows with zero row sum
        zero_rows = np.abs(Ad.sum(1)) < 1e-12 * np.abs(d)
        assert np.allclose((P @ np.ones(nc))[zero_rows], 1.0, atol=1e-14)
        # R = P^T exactly
        assert np.array_equal(lvl_sp(lv.R, n).toarray(), P.T)
        Ac_dense = P.T @ Ad @ P
        Ac = lvl_sp(nx_.A, nc).toarray()
        scale = np.abs(Ac_dense).max()
        assert np.abs(Ac - Ac_dense).max() <= 1e-14 * scale * max(1, l + 1) * 4
        if h.symmetric:
            assert np.abs(Ac - Ac.T).max() <= 1e-14 * scale
            np.linalg.cholesky(Ac)  # SPD


def test_c1_hierarchy_shape():
    h = O.Hierarchy(M.poisson2d(64))
    dims = [h.dims(l) for l in range(h.nlevels)]
    assert dims[0][:2] == (4096, 20224)
    assert dims[-1][0] <= 64 and all(d[0] > 64 for d in dims[:-1])


# --------------------------------------------------------------------------
# V-cycle
# --------------------------------------------------------------------------

def _dense_Minv(h, n):
    return np.stack([h.vcycle(e) for e in np.eye(n)], axis=1)


def test_vcycle_symmetric_and_convergent():
    A = M.poisson2d(12)
    h = O.Hierarchy(A, {"coarse_max": 10})
    assert h.nlevels >= 3
    Mi = _dense_Minv(h, A.n)
    assert np.abs(Mi - Mi.T).max() <= 1e-13 * np.abs(Mi).max()
    E = np.eye(A.n) - Mi @ A.to_dense()
    assert np.max(np.abs(np.linalg.eigvals(E))) < 1.0
    np.linalg.cholesky((Mi + Mi.T) / 2)


def test_two_level_cycle_algebraic_formula():
    A = M.poisson2d(10)
    h = O.Hierarchy(A, {"coarse_max": 40})
    assert h.nlevels == 2
    lv = h.level(0)
    n = A.n
    nc = lv.P.row_ptr.shape[0] and h.level(1).A.n
    Ad = A.to_dense()
    P = lvl_sp(lv.P, nc).toarray()
    W = np.diag((2.0 / 3.0) / np.diag(Ad))
    Ac = P.T @ Ad @ P
    S = np.eye(n) - W @ Ad
    E = S @ (np.eye(n) - P @ np.linalg.solve(Ac, P.T @ Ad)) @ S
    Minv_formula = (np.eye(n) - E) @ np.linalg.inv(Ad)
    assert np.allclose(_dense_Minv(h, n), Minv_formula, atol=1e-12)


def test_l1_jacobi_cycle_formula():
    A = M.poisson2d(8)
    h = O.Hierarchy(A, {"coarse_max": 40, "smoother": 1})
    lv = h.level(0)
    nc = h.level(1).A.n
    Ad = A.to_dense()
    P = lvl_sp(lv.P, nc).toarray()
    W = np.diag(1.0 / np.abs(Ad).sum(1))
    S = np.eye(A.n) - W @ Ad
    E = S @ (np.eye(A.n) - P @ np.linalg.solve(P.T @ Ad @ P, P.T @ Ad)) @ S
    assert np.allclose(_dense_Minv(h, A.n), (np.eye(A.n) - E) @ np.linalg.inv(Ad), atol=1e-12)


def test_coarse_direct_solve_single_level():
    A = M.poisson2d(7)  # 49 rows <= 64: one level, dense Cholesky
    h = O.Hierarchy(A)
    assert h.nlevels == 1
    b = np.random.default_rng(1).uniform(-1, 1, A.n)
    assert np.allclose(h.vcycle(b), np.linalg.solve(A.to_dense(), b), rtol=1e-13, atol=1e-14)
    C = M.convection_diffusion_upwind(3)  # 27 rows, LU with pivoting
    h = O.Hierarchy(C)
    b = b[:C.n]
    assert not h.symmetric
    assert np.allclose(h.vcycle(b), np.linalg.solve(C.to_dense(), b), rtol=1e-13, atol=1e-14)


def test_not_spd_detected():
    D = np.array([[1.0, 2.0], [2.0, 1.0]])  # symmetric indefinite
    A = M.CSR(*_dense_to_csr(D))
    with pytest.raises(O.OracleError) as e:
        O.Hierarchy(A, {"symmetric": 1})
    assert e.value.status == O.NOT_SPD


# --------------------------------------------------------------------------
# Krylov solvers
# --------------------------------------------------------------------------

@pytest.mark.parametrize("solver,maker", [
    (O.PCG, lambda: M.poisson2d(32)),
    (O.PCG, lambda: M.diffusion_fv(np.exp(np.random.default_rng(2).normal(size=(24, 24))))),
    (O.BICGSTAB, lambda: M.convection_diffusion_upwind(10)),
    (O.CG, lambda: M.poisson2d(20)),
    (O.BICGSTAB_NOPREC, lambda: M.convection_diffusion_upwind(8)),
])
def test_krylov_against_dense_solve(solver, maker):
    A = maker()
    b = np.random.default_rng(7).uniform(-1, 1, A.n)
    x, info = O.solve(A, b, {"solver": solver, "rtol": 1e-10})
    assert info.status == O.OK and info.rel_res_true <= 1e-10
    Ad = A.to_dense()
    xs = np.linalg.solve(Ad, b)
    kappa = np.linalg.cond(Ad)
    assert np.linalg.norm(x - xs) <= kappa * 1e-10 * np.linalg.norm(xs)
    assert np.linalg.norm(Ad @ x - b) <= 1.0001e-10 * np.linalg.norm(b)


def test_cg_eigenvector_rhs_one_iteration():
    s = 16
    A = M.poisson2d(s)
    t = np.arange(1, s + 1)
    v = np.outer(np.sin(2 * np.pi * t / (s + 1)), np.sin(3 * np.pi * t / (s + 1))).reshape(-1)
    lam = 4 - 2 * np.cos(3 * np.pi / (s + 1)) - 2 * np.cos(2 * np.pi / (s + 1))
    x, info = O.solve(A, v, {"solver": O.CG, "rtol": 1e-12})
    assert info.iters == 1
    assert np.allclose(x, v / lam, rtol=1e-13, atol=1e-15)


def test_zero_rhs_and_maxit_and_nan():
    A = M.poisson2d(16)
    x, info = O.solve(A, np.zeros(A.n))
    assert info.status == O.OK and info.iters == 0 and not x.any()
    b = np.random.default_rng(0).uniform(-1, 1, A.n)
    x, info = O.solve(A, b, {"max_iter": 2, "max_restarts": 0})
    assert info.status == O.MAXIT and info.iters == 2
    b[3] = np.nan
    x, info = O.solve(A, b)
    assert info.status == O.NAN


def test_paper_example1_iteration_band():
    g = json.load(open(GOLDEN))["ex1_poisson"]
    A = M.poisson_matrix(g["grid"])
    b = M.rhs_ones(A.n)
    _, info = O.solve(A, b, {"solver": O.BICGSTAB, "rtol": g["tolerance"]})
    assert info.status == O.OK and info.iters <= g["band_amg_max"]
    _, ic = O.solve(A, b, {"solver": O.BICGSTAB, "rtol": g["tolerance"], "amg_type": 1})
    assert ic.status == O.OK and ic.iters <= g["band_amg_max_classical"]
    _, info0 = O.solve(A, b, {"solver": O.BICGSTAB_NOPREC, "rtol": g["tolerance"]})
    lo, hi = g["band_unpreconditioned"]
    assert lo <= info0.iters <= hi
    assert info.iters < info0.iters


def test_bicgstab_breakdown_restarts_once_then_converges():
    """rho = r^.r vanishes at iteration 2 of this system (every quantity is a
    dyadic fraction, so the zero is exact in floating point): alpha = 1/4,
    omega = 1/2, r_1 = (-1/8, -1/8, 1/4) with r^ = b = (1, 1, 1).  The method
    restarts once from x_1 with r^ = r_1 and then converges to A^-1 b; the
    iteration that broke down before its products is not counted."""
    D = np.array([[3.0, 0.0, 3.0], [0.0, 4.0, -1.0], [1.0, 0.0, 2.0]])
    A = M.CSR(*_dense_to_csr(D))
    b = np.ones(3)
    x, info = O.solve(A, b, {"solver": O.BICGSTAB_NOPREC, "rtol": 1e-12})
    # without the restart the solve would end in BREAKDOWN at iteration 2
    assert info.status == O.OK, info
    assert np.allclose(x, np.linalg.solve(D, b), rtol=0, atol=1e-14)
    assert info.iters >= 2  # one iteration before the breakdown, at least one after the restart


def test_bicgstab_second_breakdown_returns_breakdown():
    """r^.A b = 0 for b = (1, 1): alpha's denominator vanishes at the first
    iteration, and again after the one restart (x is still 0, so r^ = r = b);
    the second breakdown ends the solve with BREAKDOWN, x untouched."""
    D = np.array([[1.0, -2.0], [0.0, 1.0]])
    A = M.CSR(*_dense_to_csr(D))
    x, info = O.solve(A, np.ones(2), {"solver": O.BICGSTAB_NOPREC})
    assert info.status == O.BREAKDOWN and info.iters == 2
    assert not x.any()


# --------------------------------------------------------------------------
# Adjoint (Eq. 1-2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("maker", [lambda: M.poisson2d(12), lambda: M.convection_diffusion_upwind(6)])
def test_adjoint_against_dense(maker):
    A = maker()
    rng = np.random.default_rng(11)
    b = rng.uniform(-1, 1, A.n)
    g = rng.uniform(-1, 1, A.n)
    cfg = {"solver": O.PCG if A.n == 144 else O.BICGSTAB, "rtol": 1e-13}
    h = O.Hierarchy(A, cfg)
    x, _ = h.solve(b)
    lam, dA, info = h.adjoint(x, g, A.nnz)
    Ad = A.to_dense()
    lam_ref = np.linalg.solve(Ad.T, g)
    assert np.allclose(lam, lam_ref, rtol=1e-10, atol=1e-12)
    rows = A.row_of()
    assert np.allclose(dA, -lam_ref[rows] * np.linalg.solve(Ad, b)[A.col_idx], rtol=1e-9, atol=1e-12)


def test_adjoint_central_fd_on_values():
    A = M.convection_diffusion_upwind(5)
    rng = np.random.default_rng(4)
    b = rng.uniform(-1, 1, A.n)
    xt = rng.uniform(-1, 1, A.n)
    cfg = {"solver": O.BICGSTAB, "rtol": 1e-13}

    def loss(vals, bb):
        x, info = O.solve(M.CSR(A.row_ptr, A.col_idx, vals), bb, cfg)
        return np.sum((x - xt) ** 2), x

    L0, x = loss(A.values, b)
    h = O.Hierarchy(A, cfg)
    lam, dA, _ = h.adjoint(x, 2 * (x - xt), A.nnz)
    eps = 1e-5
    for _ in range(3):
        v = rng.normal(size=A.nnz)
        fd = (loss(A.values + eps * v, b)[0] - loss(A.values - eps * v, b)[0]) / (2 * eps)
        assert dA @ v == pytest.approx(fd, rel=1e-5)
        u = rng.normal(size=A.n)
        fdb = (loss(A.values, b + eps * u)[0] - loss(A.values, b - eps * u)[0]) / (2 * eps)
        assert lam @ u == pytest.approx(fdb, rel=1e-5)


def test_paper_example2_gradient_descent():
    g = json.load(open(GOLDEN))["ex2_tridiagonal_inverse"]
    n = g["n"]
    b = M.rhs_ones(n)
    cfg = {"solver": O.PCG, "rtol": 1e-12}
    x_t, _ = O.solve(M.tridiagonal_matrix(n, g["true_diag"]), b, cfg)
    x_t_dense = np.linalg.solve(M.tridiagonal_matrix(n, g["true_diag"]).to_dense(), b)
    d = d_ref = g["init_diag"]
    d_at_bound = None
    for step in range(g["max_iters"]):
        A = M.tridiagonal_matrix(n, d)
        h = O.Hierarchy(A, cfg)
        x, _ = h.solve(b)
        lam, dA, _ = h.adjoint(x, 2 * (x - x_t), A.nnz)
        grad = dA[A.row_of() == A.col_idx].sum()  # d enters every diagonal entry
        # closed form on the exact (dense) trajectory: dL/dd = -lam . x
        Ad = M.tridiagonal_matrix(n, d_ref).to_dense()
        xr = np.linalg.solve(Ad, b)
        grad_ref = -np.linalg.solve(Ad.T, 2 * (xr - x_t_dense)) @ xr
        assert grad == pytest.approx(grad_ref, rel=1e-7, abs=1e-12)
        d -= g["lr"] * grad
        d_ref -= g["lr"] * grad_ref
        if step + 1 == g["steps_upper_bound"]:
            d_at_bound = d
        if abs(grad) < g["grad_tol"]:
            assert abs(grad_ref) < 1.01 * g["grad_tol"]
            break
    assert abs(d_at_bound - g["true_diag"]) < g["recover_abs_tol"]
    assert d == pytest.approx(g["true_diag"], abs=1e-3)


def test_symmetric_detection():
    assert O.Hierarchy(M.poisson2d(10)).symmetric
    assert not O.Hierarchy(M.convection_diffusion_upwind(5)).symmetric
    A = M.poisson2d(10)
    v = A.values.copy()
    v[1] = np.nextafter(v[1], 0)  # break bitwise symmetry of one pair
    assert not O.Hierarchy(M.CSR(A.row_ptr, A.col_idx, v)).symmetric


# --------------------------------------------------------------------------
# Numeric re-setup with the hierarchy's structure kept (Sec. 2.1 caching)
# --------------------------------------------------------------------------

def _same_hierarchy(h1, h2):
    assert h1.nlevels == h2.nlevels
    for l in range(h1.nlevels):
        a, b = h1.level(l), h2.level(l)
        for m1, m2 in [(a.A, b.A)] + ([(a.P, b.P), (a.R, b.R)] if l < h1.nlevels - 1 else []):
            assert np.array_equal(m1.row_ptr, m2.row_ptr) and np.array_equal(m1.col_idx, m2.col_idx)
            assert np.array_equal(m1.values.view(np.int64), m2.values.view(np.int64))
        if l < h1.nlevels - 1:
            assert np.array_equal(a.agg, b.agg)


@pytest.mark.parametrize("maker", [lambda: M.poisson2d(20), lambda: M.diffusion3d_grf(N=10).A,
                                   lambda: M.convection_diffusion_upwind(8)])
def test_resetup_same_values_is_setup(maker):
    A = maker()
    h = O.Hierarchy(A, {"coarse_max": 16})
    _same_hierarchy(h, h.resetup(A.values))


@pytest.mark.parametrize("maker", [lambda: M.poisson2d(20), lambda: M.diffusion3d_grf(N=10).A])
def test_resetup_doubled_values(maker):
    """Doubling every value is exact: D^-1 A and the strength test are unchanged,
    so P and the aggregates stay, every coarse operator doubles exactly, and the
    result equals a fresh setup of 2A."""
    A = maker()
    h = O.Hierarchy(A, {"coarse_max": 16})
    A2 = M.CSR(A.row_ptr, A.col_idx, 2.0 * A.values)
    hr = h.resetup(A2.values)
    _same_hierarchy(hr, O.Hierarchy(A2, {"coarse_max": 16}))
    for l in range(h.nlevels):
        assert np.array_equal(hr.level(l).A.values, 2.0 * h.level(l).A.values)
        if l < h.nlevels - 1:
            assert np.array_equal(hr.level(l).P.values, h.level(l).P.values)


def test_resetup_new_coefficients_keeps_structure_and_is_galerkin():
    """New log-conductivities: the aggregates and patterns are the old ones, the
    values follow the prolongator and Galerkin definitions (dense check), and
    the cycle still preconditions PCG to the tolerance."""
    rng = np.random.default_rng(7)
    A = M.diffusion_fv(np.exp(rng.normal(size=(18, 18))))
    Anew = M.diffusion_fv(np.exp(rng.normal(size=(18, 18))))
    assert np.array_equal(A.col_idx, Anew.col_idx)
    h = O.Hierarchy(A, {"coarse_max": 8})
    hr = h.resetup(Anew.values)
    assert hr.nlevels == h.nlevels >= 3
    for l in range(h.nlevels - 1):
        lv, nx_ = hr.level(l), hr.level(l + 1)
        assert np.array_equal(lv.agg, h.level(l).agg)
        assert np.array_equal(lv.P.col_idx, h.level(l).P.col_idx)
        n, nc = lv.A.n, nx_.A.n
        Ad = lvl_sp(lv.A, n).toarray()
        T = np.zeros((n, nc))
        T[np.arange(n), lv.agg] = 1.0
        d = np.diag(Ad)
        rho = np.max(np.abs(Ad).sum(1) / np.abs(d))
        Pd = (np.eye(n) - (4.0 / 3.0) / rho * (Ad / d[:, None])) @ T
        P = lvl_sp(lv.P, nc).toarray()
        assert np.allclose(P, Pd, rtol=0, atol=1e-14)
        Ac_dense = P.T @ Ad @ P
        assert np.abs(lvl_sp(nx_.A, nc).toarray() - Ac_dense).max() <= 1e-13 * np.abs(Ac_dense).max()
    b = rng.uniform(-1, 1, A.n)
    x, info = hr.solve(b)
    assert info.status == 0
    assert np.linalg.norm(to_sp(Anew) @ x - b) <= 1e-8 * np.linalg.norm(b) * 1.0001


# ---------------------------------------------------------------------------
# Transposed-hierarchy reuse for the nonsymmetric adjoint
# ---------------------------------------------------------------------------

def test_transposed_hierarchy_is_exact_transpose_and_galerkin_for_At():
    """or_transposed keeps A's aggregates, P and R and transposes every level
    operator exactly; since R = P^T each transposed level is the Galerkin
    product of the level above it with A's P (dense check)."""
    A = M.convection_diffusion_upwind(10)
    h = O.Hierarchy(A, {"solver": 1, "coarse_max": 16})
    t = h.transposed()
    assert t.nlevels == h.nlevels >= 3 and not t.symmetric
    for l in range(h.nlevels):
        a, b = h.level(l), t.level(l)
        n = a.A.n
        Ad = lvl_sp(a.A, n).toarray()
        assert np.array_equal(lvl_sp(b.A, n).toarray(), Ad.T)  # bit for bit
        if l < h.nlevels - 1:
            assert np.array_equal(b.agg, a.agg)
            for X, Y in ((a.P, b.P), (a.R, b.R)):
                assert np.array_equal(X.row_ptr, Y.row_ptr) and np.array_equal(X.col_idx, Y.col_idx)
                assert np.array_equal(X.values, Y.values)
            nc = h.level(l + 1).A.n
            P = lvl_sp(a.P, nc).toarray()
            Gal = P.T @ Ad.T @ P
            At_next = lvl_sp(t.level(l + 1).A, nc).toarray()
            assert np.abs(At_next - Gal).max() <= 1e-13 * np.abs(Gal).max()


def test_transposed_hierarchy_of_symmetric_matrix_gives_the_same_cycle():
    """For a symmetric A the finest transposed level is A itself and the coarse
    ones equal A's up to the rounding of their Galerkin sums (which are
    symmetric in exact arithmetic only), so the cycle is A's up to rounding
    and the coarsest factor (LU in place of Cholesky)."""
    A = M.poisson2d(30)
    h = O.Hierarchy(A)
    t = h.transposed()
    assert np.array_equal(t.level(0).A.values, h.level(0).A.values)
    for l in range(1, h.nlevels):
        a, b = h.level(l).A.values, t.level(l).A.values
        assert np.array_equal(t.level(l).A.col_idx, h.level(l).A.col_idx)
        assert np.abs(b - a).max() <= 1e-14 * np.abs(a).max()
    r = np.random.default_rng(2).uniform(-1, 1, A.n)
    z, zt = h.vcycle(r), t.vcycle(r)
    assert np.linalg.norm(zt - z) <= 1e-12 * np.linalg.norm(z)


def test_adjoint_reuse_solves_the_transposed_system():
    """With adjoint_reuse the adjoint solve runs BiCGStab on A^T with the
    transposed hierarchy: lambda satisfies A^T lambda = g to the tolerance and
    agrees with the adjoint of a hierarchy set up on A^T."""
    A = M.convection_diffusion_upwind(12)
    rng = np.random.default_rng(4)
    b, g = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    At = to_sp(A).T.tocsr()
    lams = []
    for reuse in (0, 1):
        h = O.Hierarchy(A, {"solver": 1, "adjoint_reuse": reuse, "rtol": 1e-12})
        x, _ = h.solve(b)
        lam, dA, info = h.adjoint(x, g, A.nnz)
        assert info.status == 0
        assert np.linalg.norm(At @ lam - g) <= 1e-12 * np.linalg.norm(g) * 1.0001
        rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
        assert np.array_equal(dA, -(lam[rows] * x[A.col_idx]))
        lams.append(lam)
    assert np.linalg.norm(lams[1] - lams[0]) <= 1e-9 * np.linalg.norm(lams[0])


# ---------------------------------------------------------------------------
# Classical Ruge-Stueben coarsening (amg_type = 1)
# ---------------------------------------------------------------------------

def classical_strength_dense(A):
    """The strong dependencies S_i of the definition (dense, for small A)."""
    Ad = to_sp(A).toarray()
    S = np.zeros_like(Ad, dtype=bool)
    for i in range(A.n):
        off = -np.delete(Ad[i], i)
        m = off.max() if off.size else 0.0
        if m > 0:
            S[i] = -Ad[i] >= 0.25 * m
            S[i, i] = False
    return S & (Ad != 0)


@pytest.mark.parametrize("maker", [lambda: M.poisson2d(23), lambda: M.convection_diffusion_upwind(7),
                                   lambda: M.diffusion_fv(np.exp(np.random.default_rng(5).normal(size=(16, 16))))])
def test_classical_split_is_a_pmis_splitting(maker):
    """No two C points depend strongly on each other (whichever turned C
    first would have turned the other F), which for a symmetric S makes the C
    points independent; every F point that influences some point depends
    strongly on a C point (PMIS turns a point F only next to a new C point);
    the splitting is complete."""
    A = maker()
    cf, rounds = O.classical_split(A)
    S = classical_strength_dense(A)
    C = cf == 1
    assert set(np.unique(cf)) <= {0, 1} and rounds >= 1 and C.any() and (~C).any()
    assert not (S & S.T)[np.ix_(C, C)].any()
    if (S == S.T).all():
        assert not S[np.ix_(C, C)].any()
    influences = S.sum(0) > 0  # i strongly influences some point
    for i in np.where(~C & influences)[0]:
        assert S[i, C].any(), i


def test_classical_split_1d_laplacian_alternates():
    """On tridiag(-1, 2, -1) every neighbour is strong; the C points form an
    independent set and every F point sits next to a C point, so no two
    neighbours are both C and no two consecutive points are both F except
    where both have a C neighbour on their other side."""
    A = M.tridiagonal_matrix(200, 2.0)
    cf, _ = O.classical_split(A)
    c = np.where(cf == 1)[0]
    assert (np.diff(c) >= 2).all() and (np.diff(c) <= 3).all()
    assert c[0] <= 1 and c[-1] >= 198


def test_classical_interpolation_reproduces_constants_and_is_galerkin():
    """Direct interpolation: an F row of a zero-row-sum stencil sums to 1 (the
    lumped diagonal equals minus the negative off-diagonal sum), a C row is a
    unit row; the coarse operators are P^T A P (dense check)."""
    A = M.poisson2d(24)
    h = O.Hierarchy(A, {"amg_type": 1, "coarse_max": 16})
    assert h.nlevels >= 3
    lv = h.level(0)
    n, nc = lv.A.n, h.level(1).A.n
    P = lvl_sp(lv.P, nc).toarray()
    Ad = lvl_sp(lv.A, n).toarray()
    cidx = lv.agg
    assert np.array_equal(np.sort(cidx[cidx >= 0]), np.arange(nc))
    for i in range(n):
        if cidx[i] >= 0:
            assert P[i, cidx[i]] == 1.0 and np.count_nonzero(P[i]) == 1
        elif np.isclose(Ad[i].sum(), 0.0) and P[i].any():
            assert abs(P[i].sum() - 1.0) <= 1e-14
    for l in range(h.nlevels - 1):
        a, nx_ = h.level(l), h.level(l + 1)
        Pd = lvl_sp(a.P, nx_.A.n).toarray()
        Gal = Pd.T @ lvl_sp(a.A, a.A.n).toarray() @ Pd
        assert np.abs(lvl_sp(nx_.A, nx_.A.n).toarray() - Gal).max() <= 1e-13 * np.abs(Gal).max()


@pytest.mark.parametrize("maker,solver", [(lambda: M.poisson2d(40), 0),
                                          (lambda: M.diffusion_fv(np.exp(np.random.default_rng(2).normal(size=(32, 32)))), 0),
                                          (lambda: M.convection_diffusion_upwind(10), 1)])
def test_classical_amg_preconditions_krylov(maker, solver):
    A = maker()
    b = np.random.default_rng(6).uniform(-1, 1, A.n)
    h = O.Hierarchy(A, {"amg_type": 1, "solver": solver})
    x, info = h.solve(b)
    assert info.status == 0 and info.iters <= 40
    assert np.linalg.norm(to_sp(A) @ x - b) <= 1e-8 * np.linalg.norm(b) * 1.0001
    _, plain = O.Hierarchy(A, {"solver": 2 if solver == 0 else 3, "max_iter": 5000}).solve(b)
    assert info.iters < plain.iters / 2


def test_classical_resetup_keeps_splitting_and_is_galerkin():
    """Classical re-setup: the C/F map and P's pattern stay, the weights follow
    the direct-interpolation formula on the new values (same values: the same
    hierarchy), the coarse operators are P^T A P."""
    rng = np.random.default_rng(8)
    A = M.diffusion_fv(np.exp(rng.normal(size=(20, 20))))
    Anew = M.diffusion_fv(np.exp(rng.normal(size=(20, 20))))
    h = O.Hierarchy(A, {"amg_type": 1, "coarse_max": 8})
    same = h.resetup(A.values)
    for l in range(h.nlevels):
        assert np.array_equal(same.level(l).A.values, h.level(l).A.values)
    hr = h.resetup(Anew.values)
    assert hr.nlevels == h.nlevels >= 3
    for l in range(h.nlevels - 1):
        lv, nx_ = hr.level(l), hr.level(l + 1)
        assert np.array_equal(lv.agg, h.level(l).agg)
        assert np.array_equal(lv.P.col_idx, h.level(l).P.col_idx)
        n, nc = lv.A.n, nx_.A.n
        Ad = lvl_sp(lv.A, n).toarray()
        P = lvl_sp(lv.P, nc).toarray()
        cidx = lv.agg
        for i in range(n):
            if cidx[i] >= 0:
                assert P[i, cidx[i]] == 1.0
                continue
            Ci = np.where(P[i] != 0)[0]
            if Ci.size == 0:
                continue
            fine = np.array([np.where(cidx == c)[0][0] for c in Ci])
            off = np.delete(Ad[i], i)
            alpha = off[off < 0].sum() / Ad[i, fine].sum()
            d = Ad[i, i] + off[off > 0].sum()
            assert np.allclose(P[i, Ci], -alpha * Ad[i, fine] / d, rtol=1e-13, atol=0)
        Gal = P.T @ Ad @ P
        assert np.abs(lvl_sp(nx_.A, nc).toarray() - Gal).max() <= 1e-13 * np.abs(Gal).max()
    b = rng.uniform(-1, 1, A.n)
    x, info = hr.solve(b)
    assert info.status == 0
    assert np.linalg.norm(to_sp(Anew) @ x - b) <= 1e-8 * np.linalg.norm(b) * 1.0001


def test_threaded_build_matches_serial():
    """The threaded build (timing only: the solve phase's row loops on every
    host core, dot products in fixed chunks) solves like the serial build, to
    rounding."""
    w = M.diffusion3d_grf(N=24)
    g = np.random.default_rng(2).uniform(-1, 1, w.A.n)
    h1, h2 = O.Hierarchy(w.A), O.Hierarchy(w.A, threads=True)
    x1, i1 = h1.solve(w.b)
    x2, i2 = h2.solve(w.b)
    assert i1.status == i2.status == O.OK and i1.iters == i2.iters
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)
    l1, d1, _ = h1.adjoint(x1, g, w.A.nnz)
    l2, d2, _ = h2.adjoint(x2, g, w.A.nnz)
    assert np.linalg.norm(l1 - l2) <= 1e-12 * np.linalg.norm(l1)
    assert O.threads_used() >= 1
