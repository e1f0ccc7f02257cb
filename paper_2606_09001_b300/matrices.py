"""Seeded synthetic sparse systems (CSR, int32 indices, FP64 values).

These generators play the role of the paper's ``jaxamg.matrices`` helpers
(``poisson_matrix``, ``tridiagonal_matrix``, ``rhs_ones``; Sec. 3.1-3.2) and
build the PDE workloads the solver is measured on: a 2D 5-point Poisson
problem, 3D/2D cell-centred variable-coefficient diffusion, a batch of
independent Poisson systems and a 3D upwind convection-diffusion operator.

They hold no part of the solver's arithmetic: only numpy array assembly and
numpy PCG64 random draws.  The same arrays feed the CUDA path and the CPU
oracle, so neither side replicates a random number generator.

Orderings are lexicographic with x fastest: ``i = x + s*y`` in 2D and
``i = x + N*y + N*N*z`` in 3D.  Dirichlet boundary rows are eliminated, so
every row keeps its diagonal and the columns of a row are strictly
ascending.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1000  # workload k (0-based) draws from PCG64(SEED_BASE + k)


@dataclass
class CSR:
    """A square CSR matrix: int32 row_ptr[n+1], int32 col_idx[nnz], f64 values[nnz]."""

    row_ptr: np.ndarray
    col_idx: np.ndarray
    values: np.ndarray

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col_idx] = self.values
        return d

    def row_of(self) -> np.ndarray:
        """Row index of every stored entry (length nnz)."""
        return np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.row_ptr))


@dataclass
class Workload:
    """One synthetic system (or batch of systems) with its right-hand side(s)."""

    name: str
    A: CSR
    b: np.ndarray  # (n,) or, for a batch, (n, nrhs) row-interleaved
    extra: dict = field(default_factory=dict)


def _stencil_csr(n: int, offsets: np.ndarray, cols: np.ndarray, vals: np.ndarray,
                 mask: np.ndarray) -> CSR:
    """Compress an (n, k) table of candidate entries into CSR.

    ``cols``/``vals``/``mask`` have shape (n, k) with the k candidate columns of
    each row already in ascending order; entries with ``mask`` False are dropped.
    """
    del offsets
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz exceeds the int32 index range")
    return CSR(row_ptr.astype(np.int32),
               cols[mask].astype(np.int32),
               np.ascontiguousarray(vals[mask], dtype=np.float64))


# --------------------------------------------------------------------------
# Constant-coefficient stencils (paper examples, Sec. 3.1 and 3.2)
# --------------------------------------------------------------------------

def tridiagonal_matrix(n: int, diagonal_value: float = 2.0, off_value: float = -1.0) -> CSR:
    """tridiag(off, d, off) of size n (the Toeplitz system of Sec. 3.2 and 3.3)."""
    i = np.arange(n)
    cols = np.stack([i - 1, i, i + 1], axis=1)
    vals = np.empty((n, 3))
    vals[:, 0] = off_value
    vals[:, 1] = diagonal_value
    vals[:, 2] = off_value
    mask = (cols >= 0) & (cols < n)
    return _stencil_csr(n, None, cols, vals, mask)


def poisson2d(s: int) -> CSR:
    """Unscaled 5-point Laplacian [-1; -1 4 -1; -1] on an s x s interior grid."""
    n = s * s
    i = np.arange(n, dtype=np.int64)
    x, y = i % s, i // s
    cols = np.stack([i - s, i - 1, i, i + 1, i + s], axis=1)
    vals = np.tile(np.array([-1.0, -1.0, 4.0, -1.0, -1.0]), (n, 1))
    mask = np.stack([y > 0, x > 0, np.ones(n, bool), x < s - 1, y < s - 1], axis=1)
    return _stencil_csr(n, None, cols, vals, mask)


def poisson_matrix(s: int) -> CSR:
    """Same as :func:`poisson2d` (the name the paper's examples use)."""
    return poisson2d(s)


def poisson3d(N: int) -> CSR:
    """Unscaled 7-point Laplacian on an N^3 interior grid."""
    n = N ** 3
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % N, (i // N) % N, i // (N * N)
    offs = [-N * N, -N, -1, 0, 1, N, N * N]
    cols = np.stack([i + o for o in offs], axis=1)
    vals = np.tile(np.array([-1.0, -1.0, -1.0, 6.0, -1.0, -1.0, -1.0]), (n, 1))
    mask = np.stack([z > 0, y > 0, x > 0, np.ones(n, bool), x < N - 1, y < N - 1, z < N - 1], axis=1)
    return _stencil_csr(n, None, cols, vals, mask)


def rhs_ones(n: int) -> np.ndarray:
    return np.ones(n)


# --------------------------------------------------------------------------
# Cell-centred finite-volume diffusion  -div(k grad u) = f
# --------------------------------------------------------------------------

def diffusion_fv(k: np.ndarray) -> CSR:
    """Cell-centred FV operator for -div(k grad u) on the unit square/cube.

    ``k`` has shape (N, N) or (N, N, N) (indexed [y, x] / [z, y, x]).  The
    equation is multiplied through by h^2, so an interior face between cells i
    and j has coefficient c = 2 k_i k_j / (k_i + k_j) (harmonic mean) and a
    boundary face (homogeneous Dirichlet, ghost value at distance h/2) has
    c = 2 k_i.  Row i: A_ii = sum of its face coefficients, A_ij = -c_ij.
    """
    k = np.asarray(k, dtype=np.float64)
    dim = k.ndim
    N = k.shape[0]
    kf = k.reshape(-1)
    n = kf.size
    i = np.arange(n, dtype=np.int64)
    coords = []
    stride = 1
    for _ in range(dim):
        coords.append((i // stride) % N)
        stride *= N
    strides = [N ** d for d in range(dim)]  # x, y, (z)
    # candidate neighbours in ascending column order: -z, -y, -x, self, +x, +y, +z
    neg = [(-strides[d], d) for d in reversed(range(dim))]
    pos = [(strides[d], d) for d in range(dim)]
    cand = neg + [(0, -1)] + pos
    cols = np.empty((n, len(cand)), dtype=np.int64)
    vals = np.zeros((n, len(cand)))
    mask = np.ones((n, len(cand)), dtype=bool)
    diag = np.zeros(n)
    dcol = len(neg)
    for c, (off, d) in enumerate(cand):
        cols[:, c] = i + off
        if off == 0:
            continue
        inside = coords[d] > 0 if off < 0 else coords[d] < N - 1
        mask[:, c] = inside
        j = np.where(inside, i + off, i)
        kj = kf[j]
        face = np.where(inside, 2.0 * kf * kj / (kf + kj), 2.0 * kf)
        vals[:, c] = np.where(inside, -face, 0.0)
        diag += face
    vals[:, dcol] = diag
    return _stencil_csr(n, None, cols, vals, mask)


def grf_log_k(N: int, dim: int, sigma: float, ell: float, rng: np.random.Generator,
              n_features: int = 2048) -> np.ndarray:
    """Gaussian random field with squared-exponential covariance, sampled by
    random Fourier features at the cell centres of an N^dim grid:

        g(x) = sigma * sqrt(2/M) * sum_m cos(w_m . x + phi_m),
        w_m ~ N(0, ell^-2 I),  phi_m ~ U[0, 2 pi).

    Evaluated separably: cos(w.x + phi) = Re(e^{i phi} prod_d e^{i w_d x_d}).
    Returns g with shape (N,)*dim indexed [z, y, x] / [y, x].
    """
    M = n_features
    w = rng.normal(0.0, 1.0 / ell, size=(M, dim))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=M)
    h = 1.0 / N
    centres = (np.arange(N) + 0.5) * h
    E = [np.exp(1j * np.outer(w[:, d], centres)) for d in range(dim)]  # (M, N) each
    base = np.exp(1j * phi)[:, None] * E[0]  # (M, N_x)
    if dim == 2:
        g = np.real(E[1].T @ base)  # [y, x]
    else:
        g = np.empty((N, N, N))
        for zi in range(N):
            zy = (E[2][:, zi][:, None] * E[1])  # (M, N_y)
            g[zi] = np.real(zy.T @ base)  # [y, x]
    return sigma * np.sqrt(2.0 / M) * g


# --------------------------------------------------------------------------
# Upwind convection-diffusion (nonsymmetric)
# --------------------------------------------------------------------------

def convection_diffusion_upwind(N: int, peclet=(10.0, 5.0, 2.5)) -> CSR:
    """Vertex-centred 7-point first-order upwind operator on an N^3 interior
    grid, normalised by eps/h^2: diagonal 6 + sum_d Pe_d, upwind neighbour
    (at -e_d, velocity components positive) -(1 + Pe_d), downwind neighbour -1.
    With Pe = (10, 5, 2.5) every entry is an exact binary fraction."""
    n = N ** 3
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % N, (i // N) % N, i // (N * N)
    pe_x, pe_y, pe_z = peclet
    offs = [-N * N, -N, -1, 0, 1, N, N * N]
    cols = np.stack([i + o for o in offs], axis=1)
    row = np.array([-(1.0 + pe_z), -(1.0 + pe_y), -(1.0 + pe_x), 6.0 + pe_x + pe_y + pe_z,
                    -1.0, -1.0, -1.0])
    vals = np.tile(row, (n, 1))
    mask = np.stack([z > 0, y > 0, x > 0, np.ones(n, bool), x < N - 1, y < N - 1, z < N - 1], axis=1)
    return _stencil_csr(n, None, cols, vals, mask)


# --------------------------------------------------------------------------
# Block-diagonal batches
# --------------------------------------------------------------------------

def block_diag(blocks: list[CSR]) -> tuple[CSR, np.ndarray]:
    """Concatenate square CSR blocks into one block-diagonal CSR.

    Returns (A, sys_off) where system s owns rows sys_off[s]:sys_off[s+1]."""
    sizes = np.array([b.n for b in blocks], dtype=np.int64)
    sys_off = np.zeros(len(blocks) + 1, dtype=np.int64)
    np.cumsum(sizes, out=sys_off[1:])
    nnzs = np.array([b.nnz for b in blocks], dtype=np.int64)
    nnz_off = np.zeros(len(blocks) + 1, dtype=np.int64)
    np.cumsum(nnzs, out=nnz_off[1:])
    if nnz_off[-1] >= 2**31 or sys_off[-1] >= 2**31:
        raise ValueError("batch exceeds the int32 index range")
    row_ptr = np.empty(int(sys_off[-1]) + 1, dtype=np.int64)
    col = np.empty(int(nnz_off[-1]), dtype=np.int64)
    val = np.empty(int(nnz_off[-1]))
    for s, b in enumerate(blocks):
        row_ptr[sys_off[s]:sys_off[s + 1]] = b.row_ptr[:-1].astype(np.int64) + nnz_off[s]
        col[nnz_off[s]:nnz_off[s + 1]] = b.col_idx.astype(np.int64) + sys_off[s]
        val[nnz_off[s]:nnz_off[s + 1]] = b.values
    row_ptr[-1] = nnz_off[-1]
    return CSR(row_ptr.astype(np.int32), col.astype(np.int32), val), sys_off.astype(np.int32)


# --------------------------------------------------------------------------
# The five measured workloads
# --------------------------------------------------------------------------

def poisson2d_64(seed: int = SEED_BASE + 0, s: int = 64) -> Workload:
    """2D 5-point Poisson, 64x64 interior grid (n = 4096), b ~ U[-1, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = poisson2d(s)
    b = rng.uniform(-1.0, 1.0, size=A.n)
    return Workload(f"poisson2d_{s}x{s}", A, b, {"s": s})


def diffusion3d_grf(seed: int = SEED_BASE + 1, N: int = 128, sigma: float = 1.0,
                    ell: float = 0.1) -> Workload:
    """3D 7-point variable-coefficient diffusion on N^3 cells, log k a GRF
    (sigma 1, correlation length 0.1), harmonic faces, f ~ U[-1, 1] (times h^2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = grf_log_k(N, 3, sigma, ell, rng)
    k = np.exp(g)
    A = diffusion_fv(k)
    h = 1.0 / N
    b = rng.uniform(-1.0, 1.0, size=A.n) * (h * h)
    return Workload(f"diffusion3d_grf_{N}^3", A, b, {"N": N, "log_k": g})


def diffusion2d_logk(seed: int = SEED_BASE + 2, N: int = 512) -> Workload:
    """Differentiable 2D diffusion on N x N cells: per-cell log k ~ N(0, 1),
    b ~ U[-1, 1], a seeded target x_target ~ U[-1, 1]; loss ||x - x_target||^2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.normal(0.0, 1.0, size=(N, N))
    b = rng.uniform(-1.0, 1.0, size=N * N)
    x_target = rng.uniform(-1.0, 1.0, size=N * N)
    A = diffusion_fv(np.exp(theta))
    return Workload(f"diffusion2d_logk_{N}^2", A, b, {"N": N, "theta": theta, "x_target": x_target})


def batched_poisson2d(seed: int = SEED_BASE + 3, nsys: int = 256, s_min: int = 32,
                      s_max: int = 256, nrhs: int = 8) -> Workload:
    """nsys independent 2D Poisson systems with sides ~ U{s_min..s_max},
    nrhs RHS each ~ U[-1, 1], as one block-diagonal CSR; B is (n, nrhs)
    row-interleaved (B[row, r])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = rng.integers(s_min, s_max, size=nsys, endpoint=True)
    A, sys_off = block_diag([poisson2d(int(s)) for s in sides])
    B = rng.uniform(-1.0, 1.0, size=(A.n, nrhs))
    return Workload(f"batched_poisson2d_{nsys}x{nrhs}", A, B,
                    {"sides": sides, "sys_off": sys_off, "nrhs": nrhs})


def convdiff3d_upwind(seed: int = SEED_BASE + 4, N: int = 160, peclet=(10.0, 5.0, 2.5)) -> Workload:
    """Nonsymmetric 3D upwind convection-diffusion on N^3 (cell Peclet 10 along
    x, velocity (1, 0.5, 0.25)), f ~ U[-1, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = convection_diffusion_upwind(N, peclet)
    b = rng.uniform(-1.0, 1.0, size=A.n)
    return Workload(f"convdiff3d_upwind_{N}^3", A, b, {"N": N, "peclet": peclet})


def tridiagonal_1e7(n: int = 10**7, diagonal_value: float = 4.0) -> Workload:
    """The well-conditioned Toeplitz system the paper times its unpreconditioned
    CG and BiCGStab on (Sec. 4, Fig. 2): tridiag(-1, d, -1) with n = 10^7 and
    b = ones; d = 4 is the example's true diagonal (Sec. 3.2), recovered from
    d = 10 by the optimisation loop."""
    A = tridiagonal_matrix(n, diagonal_value)
    return Workload(f"tridiagonal_{n}", A, rhs_ones(n), {"diag": diagonal_value, "init_diag": 10.0})

