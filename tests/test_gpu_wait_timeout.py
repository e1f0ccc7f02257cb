"""The bounded device waits run out cleanly.

amg_test_arm_wait_timeout arms a one-shot control that withholds one
arrival in the next solve-phase launch: 16 bytes of a bulk-copy stage that
no copy delivers (the streaming kernels' mbarrier waits), or every
grid-barrier arrival of one CTA of the cooperative coarse launch.  The waits
give up after a short limit and set the error flag; the solve returns
AMG_ERR_CUDA with the wait named, and the next solve on the same handle runs
normally and gives the same bits as before.  Nothing here faults or hangs a
GPU: every wait involved is bounded, and a withheld arrival is the only
thing missing."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_09001_b300 import _lib, api, matrices as M

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def solver(A, cfg):
    return api.Solver(dev(A.row_ptr), dev(A.col_idx), dev(A.values), cfg)


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


def traced_names(s, fn):
    s.profile(True)
    fn()
    _, recs = s.profile_records()
    s.profile(False)
    return {r["name"] for r in recs if r["launches"] > 0}


def run_timeout_then_clean(A, cfg, kind, what):
    b = np.random.default_rng(3).uniform(-1, 1, A.n)
    s = solver(A, cfg)
    x0, i0 = s.solve(dev(b))
    x0 = x0.cpu().numpy()
    assert i0.status == 0
    L = _lib.load()
    assert L.amg_test_arm_wait_timeout(s._h, kind) == 0
    with pytest.raises(api.AMGError) as e:
        s.solve(dev(b))
    assert e.value.code == _lib.AMG_ERR_CUDA
    assert what in str(e.value), str(e.value)
    x1, i1 = s.solve(dev(b))  # the next solve starts clean
    assert i1.status == 0 and i1.iters == i0.iters
    assert same_bits(x1.cpu().numpy(), x0)
    return s, b, x0


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_bulk_copy_wait_runs_out_then_next_solve_is_clean(precision):
    A = M.diffusion3d_grf(N=33).A  # 35,937 rows: the finest level's passes stream
    # sliced-ELL tiles: a bulk-copy ring (the direct layout has no waits)
    cfg = {"precision": precision, "layout": "SLICED_ELL"}
    s, b, x0 = run_timeout_then_clean(A, cfg, _lib.AMG_TEST_WITHHOLD_COPY, "bulk-copy")
    xt, _ = O.Hierarchy(A, {"rtol": 1e-13}).solve(b)
    assert np.linalg.norm(x0 - xt) <= 1e-7 * np.linalg.norm(xt)
    s.close()


def test_grid_barrier_wait_runs_out_then_next_solve_is_clean():
    # 16129 rows -> 2295 -> dense 197: the cooperative launch takes level 1
    # and the dense end
    A = M.poisson2d(127)
    cfg = {"fuse_coarse": 2}
    r = dev(np.random.default_rng(5).uniform(-1, 1, A.n))
    with solver(A, cfg) as s:
        assert "mid" in traced_names(s, lambda: s.vcycle(r))
    s, b, x0 = run_timeout_then_clean(A, cfg, _lib.AMG_TEST_WITHHOLD_BARRIER, "grid-barrier")
    xt, _ = O.Hierarchy(A, {"rtol": 1e-13}).solve(b)
    assert np.linalg.norm(x0 - xt) <= 1e-7 * np.linalg.norm(xt)
    s.close()


def test_arm_rejects_unknown_kind():
    A = M.poisson2d(20)
    with solver(A, {}) as s:
        L = _lib.load()
        assert L.amg_test_arm_wait_timeout(s._h, 7) == _lib.AMG_ERR_ARG
        assert L.amg_test_arm_wait_timeout(None, 1) == _lib.AMG_ERR_ARG
        assert L.amg_test_arm_wait_timeout(s._h, 0) == 0
