"""amg_cg_solve_noalloc: the solve for callers that may not allocate device
memory while they run (a framework that owns all device memory and only
hands an operator its planned buffers, or a loop where a cudaMalloc would
stall every stream).  It must give what amg_solve gives with the same
unpreconditioned CG, call after call, although every call reuses one fixed
device work array, and it must agree with the FP64 CPU oracle's CG.  This
file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_09001_b300 import _lib, api, matrices as M

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [("poisson2d_40", lambda: M.poisson2d(40)),
         ("tridiag_1000", lambda: M.tridiagonal_matrix(1000, 2.5)),
         ("logk2d_32", lambda: M.diffusion2d_logk(N=32).A)]


@pytest.mark.parametrize("name,gen", CASES)
def test_noalloc_cg_matches_amg_solve_twice(name, gen):
    A = gen()
    rng = np.random.default_rng(11)
    rp, ci, v = dev(A.row_ptr), dev(A.col_idx), dev(A.values)
    with api.Solver(rp, ci, v, {"solver": "CG", "max_iter": 5000}) as s:
        for call in range(2):  # two calls in a row, each against the handle's solve
            b = dev(rng.uniform(-1, 1, A.n))
            x_ref, info_ref = s.solve(b)
            x, info = api.cg_solve_noalloc(rp, ci, v, b, max_iter=5000)
            torch.cuda.synchronize()
            assert info_ref.status == 0 and info.status == 0, (call, info)
            assert info.rel_res_true <= 1e-8
            assert abs(info.iters - info_ref.iters) <= 2, (info.iters, info_ref.iters)
            xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
            assert np.linalg.norm(xn - xr) <= 1e-7 * np.linalg.norm(xr)
            assert np.abs(xn - xr).max() <= 1e-7 * np.abs(xr).max()


@pytest.mark.parametrize("name,gen", CASES)
def test_noalloc_cg_matches_oracle(name, gen):
    """Against the oracle's unpreconditioned CG: iterations within 2 of the
    oracle's at the same tolerance, and the solution within 1e-7 of a tight
    oracle solve, in norm and entry by entry."""
    A = gen()
    b = np.random.default_rng(21).uniform(-1, 1, A.n)
    _, io = O.solve(A, b, {"solver": O.CG, "max_iter": 5000})
    xt, it = O.solve(A, b, {"solver": O.CG, "max_iter": 20000, "rtol": 1e-13})
    assert io.status == O.OK and it.status == O.OK
    x, info = api.cg_solve_noalloc(dev(A.row_ptr), dev(A.col_idx), dev(A.values), dev(b), max_iter=5000)
    x = x.cpu().numpy()
    assert info.status == 0 and info.rel_res_true <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    assert np.linalg.norm(x - xt) <= 1e-7 * np.linalg.norm(xt)
    assert np.abs(x - xt).max() <= 1e-7 * np.abs(xt).max()


def test_noalloc_second_call_takes_no_device_memory():
    """The fixed work array is committed by the first call on a device; a
    later call leaves the device's free memory unchanged."""
    A = M.poisson2d(64)
    rp, ci, v = dev(A.row_ptr), dev(A.col_idx), dev(A.values)
    b = dev(np.random.default_rng(4).uniform(-1, 1, A.n))
    x = torch.empty(A.n, dtype=torch.float64, device="cuda")
    L = _lib.load()
    info = _lib.AmgInfo()

    def call():
        return L.amg_cg_solve_noalloc(A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), b.data_ptr(),
                                      x.data_ptr(), 1e-8, 5000, None, ctypes.byref(info))

    assert call() == 0  # warm-up: may load the module and commit the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert call() == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert info.status == 0 and info.rel_res_true <= 1e-8


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = _lib.load()
    small = torch.zeros(4, dtype=torch.float64, device="cuda")
    idx = torch.zeros(4, dtype=torch.int32, device="cuda")
    n = _lib.AMG_NOALLOC_MAX_N + 1
    rc = L.amg_cg_solve_noalloc(n, n, idx.data_ptr(), idx.data_ptr(), small.data_ptr(), small.data_ptr(),
                                small.data_ptr(), 1e-8, 10, None, None)
    assert rc == _lib.AMG_ERR_UNSUPPORTED
    assert str(_lib.AMG_NOALLOC_MAX_N) in _lib.last_error()


def test_noalloc_zero_rhs_and_host_arrays():
    A = M.poisson2d(8)
    rp, ci, v = dev(A.row_ptr), dev(A.col_idx), dev(A.values)
    x, info = api.cg_solve_noalloc(rp, ci, v, torch.zeros(A.n, dtype=torch.float64, device="cuda"))
    assert info.status == 0 and info.iters == 0 and not x.any()
    L = _lib.load()
    hb = np.ones(A.n)
    hx = np.empty(A.n)
    rc = L.amg_cg_solve_noalloc(A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), hb.ctypes.data,
                                hx.ctypes.data, 1e-8, 100, None, None)
    assert rc == _lib.AMG_ERR_ARG
    # pinned host memory is reachable from the GPU but is not device memory
    pb = torch.ones(A.n, dtype=torch.float64).pin_memory()
    dx = torch.empty(A.n, dtype=torch.float64, device="cuda")
    rc = L.amg_cg_solve_noalloc(A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), pb.data_ptr(),
                                dx.data_ptr(), 1e-8, 100, None, None)
    assert rc == _lib.AMG_ERR_ARG
    assert "device memory" in _lib.last_error()
