"""Python binding of the C ABI: a :class:`Solver` handle (setup once, many
solves and adjoints, Sec. 2.1 "C++/CUDA backend") and a ``solve`` entry point
in the style of the paper's ``jaxamg.solve`` with an LRU setup cache keyed
like the paper's (sparsity pattern, dimensions, precision, configuration).

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; everything is
passed to the library as raw pointers.  All arithmetic runs in the CUDA
library.
"""
from __future__ import annotations

import ctypes as C
import hashlib
from collections import OrderedDict
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from ._lib import AmgConfig, AmgInfo


class AMGError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = f"{where}: {_lib.status_string(code)} ({code})"
        detail = _lib.last_error()
        if code < 0 and detail:
            msg += f": {detail}"
        super().__init__(msg)
        self.code = code


@dataclass
class Info:
    status: int
    iters: int
    restarts: int
    nlevels: int
    rel_res_true: float
    rel_res_rec: float
    rows: list = field(default_factory=list)
    nnz: list = field(default_factory=list)
    operator_complexity: float = 0.0
    setup_ms: float = 0.0
    solve_ms: float = 0.0

    @property
    def converged(self) -> bool:
        return self.status == _lib.AMG_OK

    @staticmethod
    def from_c(ci: AmgInfo) -> "Info":
        L = ci.nlevels
        return Info(ci.status, ci.iters, ci.restarts, L, ci.rel_res_true, ci.rel_res_rec,
                    list(ci.rows[:L]), list(ci.nnz[:L]), ci.operator_complexity, ci.setup_ms, ci.solve_ms)


def make_config(config: dict | None = None) -> AmgConfig:
    """AMG configuration from a dict; unspecified keys keep the defaults.
    'solver', 'smoother', 'precision' and 'layout' accept names (e.g. "PCG",
    "MIXED", "SLICED_ELL")."""
    c = AmgConfig()
    _lib.load().amg_config_default(C.byref(c))
    for k, v in (config or {}).items():
        if k == "solver" and isinstance(v, str):
            v = _lib.SOLVERS[v.upper()]
        elif k == "smoother" and isinstance(v, str):
            v = _lib.SMOOTHERS[v.upper()]
        elif k == "precision" and isinstance(v, str):
            v = _lib.PRECISIONS[v.upper()]
        elif k == "layout" and isinstance(v, str):
            v = _lib.LAYOUTS[v.upper()]
        elif k == "amg_type" and isinstance(v, str):
            v = _lib.AMG_TYPES[v.upper()]
        if not hasattr(c, k):
            raise KeyError(f"unknown config key {k!r}")
        setattr(c, k, v)
    return c


def config_dict(c: AmgConfig) -> dict:
    return {f: getattr(c, f) for f, _ in AmgConfig._fields_}


def _ptr(a) -> int:
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _check_dtype(a, kind: str):
    want = {"i32": (torch.int32, np.int32), "f64": (torch.float64, np.float64)}[kind]
    dt = a.dtype
    if isinstance(a, torch.Tensor):
        ok = dt == want[0]
    else:
        ok = dt == want[1]
    if not ok:
        raise TypeError(f"expected {kind} array, got {dt}")


def _stream_of(*arrays) -> int:
    for a in arrays:
        if isinstance(a, torch.Tensor) and a.is_cuda:
            return torch.cuda.current_stream(a.device).cuda_stream
    return 0


class Solver:
    """A cached AMG hierarchy of one CSR matrix (amg_setup ... amg_free)."""

    def __init__(self, row_ptr, col_idx, values, config: dict | AmgConfig | None = None, stream: int | None = None):
        L = _lib.load()
        for a, k in ((row_ptr, "i32"), (col_idx, "i32"), (values, "f64")):
            _check_dtype(a, k)
        self.n = int(row_ptr.shape[0]) - 1
        self.nnz = int(col_idx.shape[0])
        self.config = config if isinstance(config, AmgConfig) else make_config(config)
        h = C.c_void_p()
        s = _stream_of(row_ptr, col_idx, values) if stream is None else stream
        rc = L.amg_setup(C.byref(self.config), self.n, self.nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(values),
                         s, C.byref(h))
        if rc != _lib.AMG_OK:
            raise AMGError(rc, "amg_setup")
        self._h = h
        self._L = L
        self.generation = 0  # counts re-setups (values the handle currently holds)

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            self._L.amg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def resetup(self, values, stream: int | None = None):
        """Numeric re-setup for new values on the same pattern: the hierarchy's
        structure (aggregates, every sparsity pattern) is kept and every value
        recomputed (Sec. 2.1's cache hit)."""
        _check_dtype(values, "f64")
        if int(values.shape[0]) != self.nnz:
            raise ValueError(f"expected {self.nnz} values, got {int(values.shape[0])}")
        s = _stream_of(values) if stream is None else stream
        rc = self._L.amg_resetup(self._h, _ptr(values), s)
        if rc != _lib.AMG_OK:
            self.close()  # a failed re-setup leaves the values partly updated
            raise AMGError(rc, "amg_resetup")
        self.generation += 1

    # -- solves --
    def solve(self, b, x=None, stream: int | None = None, info: bool = True, check: bool = False):
        """x = A^-1 b.  Returns (x, Info).  ``x`` is allocated like ``b`` if not given."""
        _check_dtype(b, "f64")
        if x is None:
            x = torch.empty_like(b) if isinstance(b, torch.Tensor) else np.empty_like(b)
        ci = AmgInfo()
        s = _stream_of(b, x) if stream is None else stream
        rc = self._L.amg_solve(self._h, _ptr(b), _ptr(x), s, C.byref(ci) if info else None)
        if rc < 0 or (check and rc != 0):
            raise AMGError(rc, "amg_solve")
        return x, (Info.from_c(ci) if info else rc)

    def adjoint(self, x, g, lam=None, dA=None, want_lambda: bool = True, want_dA: bool = True,
                stream: int | None = None, info: bool = True):
        """Adjoint of the solve (Eq. 1-2): lambda = A^-T g and
        dA[k] = -lambda[row(k)] x[col(k)].  Returns (lambda, dA, Info)."""
        _check_dtype(x, "f64")
        _check_dtype(g, "f64")
        like = g
        if want_lambda and lam is None:
            lam = torch.empty_like(like) if isinstance(like, torch.Tensor) else np.empty_like(like)
        if want_dA and dA is None:
            dA = (torch.empty(self.nnz, dtype=torch.float64, device=like.device) if isinstance(like, torch.Tensor)
                  else np.empty(self.nnz))
        ci = AmgInfo()
        s = _stream_of(x, g) if stream is None else stream
        rc = self._L.amg_adjoint(self._h, _ptr(x), _ptr(g), _ptr(lam) if want_lambda else None,
                                 _ptr(dA) if want_dA else None, s, C.byref(ci) if info else None)
        if rc < 0:
            raise AMGError(rc, "amg_adjoint")
        return lam, dA, (Info.from_c(ci) if info else rc)

    def vcycle(self, r, z=None, stream: int | None = None):
        """One application of the AMG preconditioner z = M^-1 r."""
        _check_dtype(r, "f64")
        if z is None:
            z = torch.empty_like(r) if isinstance(r, torch.Tensor) else np.empty_like(r)
        s = _stream_of(r, z) if stream is None else stream
        rc = self._L.amg_vcycle(self._h, _ptr(r), _ptr(z), s)
        if rc < 0:
            raise AMGError(rc, "amg_vcycle")
        return z

    # -- tracing --
    def profile(self, enable: bool = True):
        """Starts (or stops) per-kernel CUDA-event tracing; clears the records."""
        rc = self._L.amg_profile(self._h, 1 if enable else 0)
        if rc < 0:
            raise AMGError(rc, "amg_profile")

    def profile_product(self, reps: int = 50) -> float:
        """Microseconds per launch of the finest level's Krylov product over
        reps back-to-back launches (call after a solve)."""
        us = C.c_double()
        rc = self._L.amg_profile_product(self._h, reps, C.byref(us))
        if rc < 0:
            raise AMGError(rc, "amg_profile_product")
        return us.value

    def profile_records(self):
        """(launches, [dict(name, level, launches, ms, bytes), ...]) since the last profile() call."""
        launches, nrec = C.c_longlong(), C.c_int()
        rc = self._L.amg_profile_summary(self._h, C.byref(launches), C.byref(nrec))
        if rc < 0:
            raise AMGError(rc, "amg_profile_summary")
        out = []
        for i in range(nrec.value):
            name = C.create_string_buffer(32)
            lev, cnt, ms, by = C.c_int(), C.c_longlong(), C.c_double(), C.c_double()
            self._L.amg_profile_record(self._h, i, name, 32, C.byref(lev), C.byref(cnt), C.byref(ms), C.byref(by))
            out.append({"name": name.value.decode(), "level": lev.value, "launches": cnt.value,
                        "ms": ms.value, "bytes": by.value})
        return launches.value, out

    # -- inspection --
    def info(self) -> Info:
        ci = AmgInfo()
        rc = self._L.amg_get_info(self._h, C.byref(ci))
        if rc < 0:
            raise AMGError(rc, "amg_get_info")
        return Info.from_c(ci)

    @property
    def nlevels(self) -> int:
        return self.info().nlevels

    def level(self, l: int, which: str = "A"):
        """(row_ptr, col_idx, values, shape) of A_l, P_l or R_l as numpy arrays."""
        w = {"A": 0, "P": 1, "R": 2}[which]
        dims = (C.c_longlong * 3)()
        rc = self._L.amg_get_level(self._h, l, w, dims, None, None, None)
        if rc < 0:
            raise AMGError(rc, "amg_get_level")
        nr, nc, nnz = dims[0], dims[1], dims[2]
        rp = np.empty(nr + 1, np.int32)
        ci = np.empty(max(nnz, 1), np.int32)
        v = np.empty(max(nnz, 1))
        rc = self._L.amg_get_level(self._h, l, w, None, rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
        if rc < 0:
            raise AMGError(rc, "amg_get_level")
        return rp, ci[:nnz], v[:nnz], (nr, nc)

    def aggregates(self, l: int) -> np.ndarray:
        n = self.level(l, "A")[3][0]
        agg = np.empty(n, np.int32)
        rc = self._L.amg_get_aggregates(self._h, l, agg.ctypes.data)
        if rc < 0:
            raise AMGError(rc, "amg_get_aggregates")
        return agg

    PLAN_OPS = {"pre": 0, "P": 1, "R": 2, "post": 3, "krylov": 4}
    LAYOUT_NAMES = {0: None, 1: "CSR", 2: "WINDOWED", 3: "SLICED_ELL", 4: "ELL_DIRECT"}

    def plan(self, l: int, op: str) -> dict:
        """The streaming plan setup chose for one operator of level l (op in
        PLAN_OPS): layout name (None: row-vector kernels), rows per tile,
        threads per row, tiles, pipeline stages, and whether the product runs
        in double-FP32 arithmetic (the mixed form's Krylov product)."""
        out = (C.c_int * 6)()
        rc = self._L.amg_get_plan(self._h, l, self.PLAN_OPS[op], out)
        if rc < 0:
            raise AMGError(rc, "amg_get_plan")
        return {"layout": self.LAYOUT_NAMES[out[0]], "rows_per_tile": out[1], "threads_per_row": out[2],
                "tiles": out[3], "stages": out[4], "df": bool(out[5])}


class BatchedSolver(Solver):
    """Many independent systems, each with up to 8 right-hand sides, solved
    concurrently with one cached setup (amg_setup_batched ...
    amg_solve_batched).  The systems are passed as one block-diagonal CSR
    whose system k owns rows sys_off[k] .. sys_off[k+1]-1."""

    def __init__(self, sys_off, row_ptr, col_idx, values, config: dict | AmgConfig | None = None,
                 stream: int | None = None):
        L = _lib.load()
        for a, k in ((sys_off, "i32"), (row_ptr, "i32"), (col_idx, "i32"), (values, "f64")):
            _check_dtype(a, k)
        self.n = int(row_ptr.shape[0]) - 1
        self.nnz = int(col_idx.shape[0])
        self.nsys = int(sys_off.shape[0]) - 1
        self.config = config if isinstance(config, AmgConfig) else make_config(config)
        h = C.c_void_p()
        s = _stream_of(row_ptr, col_idx, values) if stream is None else stream
        rc = L.amg_setup_batched(C.byref(self.config), self.nsys, _ptr(sys_off), self.n, self.nnz, _ptr(row_ptr),
                                 _ptr(col_idx), _ptr(values), s, C.byref(h))
        if rc != _lib.AMG_OK:
            raise AMGError(rc, "amg_setup_batched")
        self._h = h
        self._L = L

    def solve(self, B, X=None, stream: int | None = None, info: bool = True, check: bool = False):
        """X[:, r] = A^-1 B[:, r] for every column of B (n x nrhs, nrhs <= 8)
        on every system.  Returns (X, iters [nsys, nrhs], rel_res [nsys, nrhs],
        Info)."""
        _check_dtype(B, "f64")
        if B.ndim == 1:
            B = B.reshape(-1, 1)
        nrhs = int(B.shape[1])
        if X is None:
            X = torch.empty_like(B) if isinstance(B, torch.Tensor) else np.empty_like(B)
        its = np.empty((self.nsys, nrhs), np.int32)
        rel = np.empty((self.nsys, nrhs))
        ci = AmgInfo()
        s = _stream_of(B, X) if stream is None else stream
        rc = self._L.amg_solve_batched(self._h, nrhs, _ptr(B), _ptr(X), its.ctypes.data, rel.ctypes.data, s,
                                       C.byref(ci) if info else None)
        if rc < 0 or (check and rc != 0):
            raise AMGError(rc, "amg_solve_batched")
        return X, its, rel, (Info.from_c(ci) if info else rc)

    def adjoint(self, *a, **k):
        raise AMGError(_lib.AMG_ERR_ARG, "BatchedSolver.adjoint (not provided for batches)")

    def vcycle(self, *a, **k):
        raise AMGError(_lib.AMG_ERR_ARG, "BatchedSolver.vcycle (not provided for batches)")

    def batch_level(self, l: int):
        """(system ids, row offsets, final flags) of level l."""
        ns = C.c_int()
        sys_ = np.empty(self.nsys, np.int32)
        off = np.empty(self.nsys + 1, np.int32)
        fin = np.empty(self.nsys, np.int32)
        rc = self._L.amg_batch_level(self._h, l, C.byref(ns), sys_.ctypes.data, off.ctypes.data, fin.ctypes.data)
        if rc < 0:
            raise AMGError(rc, "amg_batch_level")
        k = ns.value
        return sys_[:k], off[:k + 1], fin[:k].astype(bool)


# ---------------------------------------------------------------------------
# Setup cache and the solve entry point
# ---------------------------------------------------------------------------

def _digest(*arrays) -> str:
    h = hashlib.blake2b(digest_size=16)
    for a in arrays:
        if isinstance(a, torch.Tensor):
            a = a.detach()
            if a.is_cuda:
                a = a.cpu()
            a = a.numpy()
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


class SetupCache:
    """LRU cache of Solver handles keyed by a hash of the full sparsity
    pattern, the dimensions, the precision and the configuration (the key
    the paper's backend uses).  A hit whose values differ re-sets the cached
    hierarchy up for the new values, keeping its structure (Sec. 2.1); with
    resetup=False it builds a new hierarchy instead.  The pattern hash is
    memoised per tensor (identity and version counter); values are compared
    exactly against a stored copy on their own device."""

    def __init__(self, capacity: int = 8, resetup: bool = True):
        self.capacity = capacity
        self.resetup = resetup
        self._d: OrderedDict = OrderedDict()
        self._pattern_memo: dict = {}
        self.hits = self.misses = self.resetups = 0

    def _pattern_digest(self, row_ptr, col_idx) -> str:
        if isinstance(row_ptr, torch.Tensor) and isinstance(col_idx, torch.Tensor):
            mk = (row_ptr.data_ptr(), row_ptr._version, tuple(row_ptr.shape), str(row_ptr.device),
                  col_idx.data_ptr(), col_idx._version, tuple(col_idx.shape))
            d = self._pattern_memo.get(mk)
            if d is None:
                d = _digest(row_ptr, col_idx)
                if len(self._pattern_memo) > 64:
                    self._pattern_memo.clear()
                self._pattern_memo[mk] = d
            return d
        return _digest(row_ptr, col_idx)

    def key(self, row_ptr, col_idx, cfg: AmgConfig):
        return (self._pattern_digest(row_ptr, col_idx), int(row_ptr.shape[0]) - 1, int(col_idx.shape[0]),
                tuple(sorted(config_dict(cfg).items())))

    @staticmethod
    def _same(a, b) -> bool:
        if isinstance(a, torch.Tensor) and isinstance(b, torch.Tensor):
            return a.device == b.device and a.shape == b.shape and bool(torch.equal(a, b))
        if isinstance(a, np.ndarray) and isinstance(b, np.ndarray):
            return a.shape == b.shape and np.array_equal(a, b)
        return False

    def get(self, row_ptr, col_idx, values, cfg: AmgConfig) -> Solver:
        k = self.key(row_ptr, col_idx, cfg)
        ent = self._d.get(k)
        if ent is not None and self._same(ent[1], values):
            self._d.move_to_end(k)
            self.hits += 1
            return ent[0]
        kept = values.detach().clone() if isinstance(values, torch.Tensor) else np.array(values, copy=True)
        if ent is not None and self.resetup:
            ent[0].resetup(values)
            self._d[k] = (ent[0], kept)
            self._d.move_to_end(k)
            self.resetups += 1
            return ent[0]
        self.misses += 1
        if ent is not None:
            ent[0].close()
        s = Solver(row_ptr, col_idx, values, cfg)
        self._d[k] = (s, kept)
        self._d.move_to_end(k)
        while len(self._d) > self.capacity:
            _, (old, _) = self._d.popitem(last=False)
            old.close()
        return s

    def clear(self):
        for s, _ in self._d.values():
            s.close()
        self._d.clear()


default_cache = SetupCache()


def solve(A, b, config: dict | None = None, cache: SetupCache | None = default_cache):
    """x, info = solve(A, b, config): AMG-preconditioned Krylov solve of the
    CSR matrix A = (row_ptr, col_idx, values) (or an object with those
    attributes).  The hierarchy is cached and reused across calls."""
    rp, ci, v = (A.row_ptr, A.col_idx, A.values) if hasattr(A, "row_ptr") else A
    cfg = make_config(config)
    s = cache.get(rp, ci, v, cfg) if cache is not None else Solver(rp, ci, v, cfg)
    return s.solve(b)


def cg_solve_noalloc(row_ptr, col_idx, values, b, x=None, rtol: float = 1e-8, max_iter: int = 500,
                     stream: int | None = None):
    """Unpreconditioned CG through amg_cg_solve_noalloc: the library allocates
    no device memory for this call (it works in a fixed device array), for
    callers that may not allocate while they run.  All arrays must be CUDA
    tensors; ``x`` is allocated here only when the caller does not pass one.
    Returns (x, Info)."""
    L = _lib.load()
    for a, k in ((row_ptr, "i32"), (col_idx, "i32"), (values, "f64"), (b, "f64")):
        _check_dtype(a, k)
    if x is None:
        x = torch.empty_like(b)
    ci = AmgInfo()
    s = _stream_of(b, x) if stream is None else stream
    rc = L.amg_cg_solve_noalloc(int(row_ptr.shape[0]) - 1, int(col_idx.shape[0]), _ptr(row_ptr), _ptr(col_idx),
                                _ptr(values), _ptr(b), _ptr(x), rtol, max_iter, s, C.byref(ci))
    if rc < 0:
        raise AMGError(rc, "amg_cg_solve_noalloc")
    return x, Info.from_c(ci)
