"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python access (ctypes + numpy) to ``amg_oracle.c``, the plain single-threaded
C implementation of the smoothed-aggregation AMG hierarchy, the V(1,1)
cycle, PCG/BiCGStab and the solve adjoint (the paper's Eq. 1-2).  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library and never
imports it.

Every function here is pinned by ``tests/test_oracle.py`` against facts that
do not come from the oracle itself (closed-form eigenpairs, dense direct
solves, brute-force MIS-2 checks, an explicitly formed P^T A P, finite
differences, and the paper's worked examples).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# the same source built with -fopenmp: the solve phase's row loops on every
# host core, for timing the CPU baseline only (parity uses the serial build)
_LIB_THREADS = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

OK, MAXIT, BREAKDOWN, NOT_SPD, NAN = 0, 1, 2, 3, 4
ERR_ARG, ERR_BAD_CSR, ERR_ZERO_DIAG, ERR_STALL, ERR_OOM = -1, -2, -3, -5, -6

PCG, BICGSTAB, CG, BICGSTAB_NOPREC = 0, 1, 2, 3


def build(force: bool = False, threads: bool = False) -> str:
    """Compile amg_oracle.c into liboracle.so (gcc, no FMA contraction), or
    with threads=True into liboracle_omp.so (the same with -fopenmp)."""
    out = _LIB_THREADS if threads else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        if threads:
            cmd.insert(1, "-fopenmp")
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def threads_used() -> int:
    """Threads the threaded build's parallel loops run on (OMP_NUM_THREADS,
    else every core this process may use)."""
    env = os.environ.get("OMP_NUM_THREADS", "").split(",")[0].strip()
    if env.isdigit() and int(env) > 0:
        return int(env)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class _Config(C.Structure):
    _fields_ = [("solver", C.c_int), ("smoother", C.c_int), ("omega", C.c_double),
                ("theta", C.c_double), ("coarse_max", C.c_int), ("max_levels", C.c_int),
                ("rtol", C.c_double), ("max_iter", C.c_int), ("max_restarts", C.c_int),
                ("symmetric", C.c_int), ("adjoint_reuse", C.c_int),
                ("amg_type", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("restarts", C.c_int),
                ("rel_res_true", C.c_double), ("rel_res_rec", C.c_double)]


_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib(threads: bool = False):
    with _lock:
        if threads not in _libs:
            L = C.CDLL(build(threads=threads))
            L.or_config_default.argtypes = [C.POINTER(_Config)]
            L.or_validate.argtypes = [C.c_int, C.c_longlong, _i32p, _i32p, _f64p]
            L.or_spmv.argtypes = [C.c_int, _i32p, _i32p, _f64p, _f64p, _f64p]
            L.or_transpose.argtypes = [C.c_int, C.c_int, C.c_longlong, _i32p, _i32p, _f64p,
                                       _i32p, _i32p, _f64p]
            L.or_strength.argtypes = [C.c_int, C.c_longlong, _i32p, _i32p, _f64p, C.c_double,
                                      C.POINTER(C.POINTER(C.c_int)), C.POINTER(C.POINTER(C.c_int)),
                                      C.POINTER(C.c_longlong)]
            L.or_free_buf.argtypes = [C.c_void_p]
            L.or_fmix32.argtypes = [C.c_uint32]
            L.or_fmix32.restype = C.c_uint32
            L.or_mis2.argtypes = [C.c_int, _i32p, _i32p, C.c_int, _i32p, C.POINTER(C.c_int)]
            L.or_aggregate_roots.argtypes = [C.c_int, C.c_longlong, _i32p, _i32p, _f64p, _i32p,
                                             _i32p, _i32p, _i32p, C.POINTER(C.c_int)]
            L.or_setup.argtypes = [C.POINTER(_Config), C.c_int, C.c_longlong, _i32p, _i32p, _f64p,
                                   C.POINTER(C.c_int)]
            L.or_setup.restype = C.c_void_p
            L.or_resetup.argtypes = [C.c_void_p, _f64p, C.POINTER(C.c_int)]
            L.or_resetup.restype = C.c_void_p
            L.or_transposed.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
            L.or_classical_split.argtypes = [C.c_int, C.c_longlong, _i32p, _i32p, _f64p, _i32p,
                                             C.POINTER(C.c_int)]
            L.or_transposed.restype = C.c_void_p
            L.or_hier_free.argtypes = [C.c_void_p]
            L.or_hier_nlevels.argtypes = [C.c_void_p]
            L.or_hier_symmetric.argtypes = [C.c_void_p]
            L.or_hier_rho.argtypes = [C.c_void_p, C.c_int]
            L.or_hier_rho.restype = C.c_double
            L.or_hier_dims.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                       C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                                       C.POINTER(C.c_longlong)]
            L.or_hier_get.argtypes = [C.c_void_p, C.c_int, C.c_int, _i32p, _i32p, _f64p]
            L.or_hier_get_agg.argtypes = [C.c_void_p, C.c_int, _i32p]
            L.or_hier_strength_nnz.argtypes = [C.c_void_p, C.c_int]
            L.or_hier_strength_nnz.restype = C.c_longlong
            L.or_hier_get_strength.argtypes = [C.c_void_p, C.c_int, _i32p, _i32p]
            L.or_hier_coarse_n.argtypes = [C.c_void_p]
            L.or_vcycle.argtypes = [C.c_void_p, _f64p, _f64p]
            L.or_dense_solve.argtypes = [C.c_void_p, _f64p, _f64p]
            L.or_solve.argtypes = [C.c_void_p, _f64p, _f64p, C.POINTER(_Info)]
            L.or_adjoint.argtypes = [C.c_void_p, _f64p, _f64p, _f64p, _f64p, C.POINTER(_Info)]
            _libs[threads] = L
    return _libs[threads]


def _csr_args(A):
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(A.values, dtype=np.float64)
    return rp, ci, v


@dataclass
class Info:
    status: int
    iters: int
    restarts: int
    rel_res_true: float
    rel_res_rec: float


def default_config(**kw) -> dict:
    c = _Config()
    lib().or_config_default(C.byref(c))
    d = {f: getattr(c, f) for f, _ in _Config._fields_}
    d.update(kw)
    return d


def _make_config(cfg: dict | None) -> _Config:
    d = default_config(**(cfg or {}))
    return _Config(**d)


def validate(A) -> int:
    rp, ci, v = _csr_args(A)
    return lib().or_validate(A.n, A.nnz, rp, ci, v)


def spmv(A, x):
    rp, ci, v = _csr_args(A)
    y = np.empty(A.n)
    lib().or_spmv(A.n, rp, ci, v, np.ascontiguousarray(x, dtype=np.float64), y)
    return y


def transpose(rp, ci, v, ncols):
    nrows = rp.shape[0] - 1
    nnz = ci.shape[0]
    trp = np.empty(ncols + 1, np.int32)
    tci = np.empty(nnz, np.int32)
    tv = np.empty(nnz)
    lib().or_transpose(nrows, ncols, nnz, np.ascontiguousarray(rp, np.int32),
                       np.ascontiguousarray(ci, np.int32), np.ascontiguousarray(v, np.float64),
                       trp, tci, tv)
    return trp, tci, tv


def strength(A, theta: float = 0.08):
    rp, ci, v = _csr_args(A)
    srp, sci, snnz = C.POINTER(C.c_int)(), C.POINTER(C.c_int)(), C.c_longlong()
    st = lib().or_strength(A.n, A.nnz, rp, ci, v, theta, C.byref(srp), C.byref(sci), C.byref(snnz))
    if st:
        raise RuntimeError(f"or_strength failed: {st}")
    out_rp = np.ctypeslib.as_array(srp, shape=(A.n + 1,)).copy()
    out_ci = np.ctypeslib.as_array(sci, shape=(max(snnz.value, 1),))[: snnz.value].copy()
    lib().or_free_buf(C.cast(srp, C.c_void_p))
    lib().or_free_buf(C.cast(sci, C.c_void_p))
    return out_rp, out_ci


def fmix32(i: int) -> int:
    return int(lib().or_fmix32(i & 0xFFFFFFFF))


def mis2(srp, sci, method: str = "greedy"):
    n = srp.shape[0] - 1
    root = np.empty(n, np.int32)
    rounds = C.c_int(0)
    st = lib().or_mis2(n, np.ascontiguousarray(srp, np.int32), np.ascontiguousarray(sci, np.int32),
                       0 if method == "greedy" else 1, root, C.byref(rounds))
    if st:
        raise RuntimeError(f"or_mis2 failed: {st}")
    return root.astype(bool), rounds.value


def aggregate(A, srp, sci, root):
    rp, ci, v = _csr_args(A)
    agg = np.empty(A.n, np.int32)
    nc = C.c_int()
    st = lib().or_aggregate_roots(A.n, A.nnz, rp, ci, v, np.ascontiguousarray(srp, np.int32),
                                  np.ascontiguousarray(sci, np.int32),
                                  np.ascontiguousarray(root, np.int32), agg, C.byref(nc))
    if st:
        raise RuntimeError(f"or_aggregate_roots failed: {st}")
    return agg, nc.value


class Level:
    def __init__(self, A, P, R, agg, rho):
        self.A, self.P, self.R, self.agg, self.rho = A, P, R, agg, rho


class Hierarchy:
    """An oracle AMG hierarchy (owns C memory; freed on close/GC)."""

    def __init__(self, A, config: dict | None = None, threads: bool = False):
        """threads=True: the threaded build (solve phase on every host core;
        timing only, its dot products round differently from the serial build)."""
        self._cfg = _make_config(config)
        self._L = lib(threads)
        rp, ci, v = _csr_args(A)
        st = C.c_int()
        h = self._L.or_setup(C.byref(self._cfg), A.n, A.nnz, rp, ci, v, C.byref(st))
        self.status = st.value
        if not h:
            raise OracleError(self.status)
        self._h = C.c_void_p(h)
        self.n = A.n

    def resetup(self, values) -> "Hierarchy":
        """A new hierarchy for the same pattern with new values, keeping this
        one's aggregates (hence every sparsity pattern) and recomputing every
        value: the numeric re-setup of the cached-setup path (Sec. 2.1)."""
        st = C.c_int()
        v = np.ascontiguousarray(values, dtype=np.float64)
        h = self._L.or_resetup(self._h, v, C.byref(st))
        if not h:
            raise OracleError(st.value)
        out = Hierarchy.__new__(Hierarchy)
        out._cfg = self._cfg
        out._L = self._L
        out._h = C.c_void_p(h)
        out.status = st.value
        out.n = self.n
        return out

    def transposed(self) -> "Hierarchy":
        """The hierarchy of A^T that keeps this one's aggregates, P and R and
        transposes every level operator (the adjoint's hierarchy with
        adjoint_reuse)."""
        st = C.c_int()
        h = self._L.or_transposed(self._h, C.byref(st))
        if not h:
            raise OracleError(st.value)
        out = Hierarchy.__new__(Hierarchy)
        out._cfg = self._cfg
        out._L = self._L
        out._h = C.c_void_p(h)
        out.status = st.value
        out.n = self.n
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._L.or_hier_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nlevels(self) -> int:
        return self._L.or_hier_nlevels(self._h)

    @property
    def symmetric(self) -> bool:
        return bool(self._L.or_hier_symmetric(self._h))

    def dims(self, l):
        n, nnzA, nc, nnzP = C.c_int(), C.c_longlong(), C.c_int(), C.c_longlong()
        self._L.or_hier_dims(self._h, l, C.byref(n), C.byref(nnzA), C.byref(nc), C.byref(nnzP))
        return n.value, nnzA.value, nc.value, nnzP.value

    def level(self, l) -> Level:
        from types import SimpleNamespace
        n, nnzA, nc, nnzP = self.dims(l)

        def get(which, nrows, nnz):
            rp = np.empty(nrows + 1, np.int32)
            ci = np.empty(max(nnz, 1), np.int32)
            v = np.empty(max(nnz, 1))
            self._L.or_hier_get(self._h, l, which, rp, ci, v)
            return SimpleNamespace(row_ptr=rp, col_idx=ci[:nnz], values=v[:nnz], n=nrows, nnz=nnz)

        A = get(0, n, nnzA)
        P = R = agg = None
        if nc > 0:
            P = get(1, n, nnzP)
            R = get(2, nc, nnzP)
            agg = np.empty(n, np.int32)
            self._L.or_hier_get_agg(self._h, l, agg)
        return Level(A, P, R, agg, self._L.or_hier_rho(self._h, l))

    def strength(self, l):
        """The strength graph (row_ptr, col_idx) level l's aggregation used,
        as the setup kept it, or None (classical levels, re-setups)."""
        nnz = self._L.or_hier_strength_nnz(self._h, l)
        if nnz < 0:
            return None
        n = self.dims(l)[0]
        srp = np.empty(n + 1, np.int32)
        sci = np.empty(max(nnz, 1), np.int32)
        self._L.or_hier_get_strength(self._h, l, srp, sci)
        return srp, sci[:nnz]

    def vcycle(self, b):
        x = np.empty(self.n)
        self._L.or_vcycle(self._h, np.ascontiguousarray(b, np.float64), x)
        return x

    def solve(self, b):
        x = np.empty(self.n)
        info = _Info()
        self._L.or_solve(self._h, np.ascontiguousarray(b, np.float64), x, C.byref(info))
        return x, Info(info.status, info.iters, info.restarts, info.rel_res_true, info.rel_res_rec)

    def adjoint(self, x, g, nnz):
        lam = np.empty(self.n)
        dA = np.empty(nnz)
        info = _Info()
        self._L.or_adjoint(self._h, np.ascontiguousarray(x, np.float64),
                         np.ascontiguousarray(g, np.float64), lam, dA, C.byref(info))
        return lam, dA, Info(info.status, info.iters, info.restarts, info.rel_res_true,
                             info.rel_res_rec)


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle setup failed with status {status}")
        self.status = status


def classical_split(A):
    """The classical C/F splitting of A (strength, PMIS): (cf with 1 for C and
    0 for F, rounds)."""
    rp, ci, v = _csr_args(A)
    cf = np.empty(A.n, np.int32)
    r = C.c_int()
    st = lib().or_classical_split(A.n, A.nnz, rp, ci, v, cf, C.byref(r))
    if st:
        raise OracleError(st)
    return cf, r.value


def solve(A, b, config: dict | None = None):
    """Setup + solve; returns (x, Info)."""
    h = Hierarchy(A, config)
    try:
        return h.solve(b)
    finally:
        h.close()
