"""The integer-pipe FP64 <-> FP32 conversions of the mixed-precision form
(amg_narrow_f64, amg_widen_f32) against the GPU's own cvt instructions (what
torch's dtype casts run), bit for bit, on random bit patterns and on the edge
cases IEEE 754 singles out: signed zeros, subnormals of either format,
values next to the binary32 range, exact halfway ties, infinities, NaN."""
import numpy as np
import pytest
import torch

from paper_2606_09001_b300 import _lib

pytestmark = pytest.mark.gpu


def narrow(x):
    out = torch.empty(x.numel(), dtype=torch.float32, device=x.device)
    assert _lib.load().amg_narrow_f64(x.data_ptr(), out.data_ptr(), x.numel(), None) == 0
    torch.cuda.synchronize()
    return out


def widen(x):
    out = torch.empty(x.numel(), dtype=torch.float64, device=x.device)
    assert _lib.load().amg_widen_f32(x.data_ptr(), out.data_ptr(), x.numel(), None) == 0
    torch.cuda.synchronize()
    return out


def same_bits(a, b):
    nan = torch.isnan(a)
    assert torch.equal(nan, torch.isnan(b))
    ia = a.view(torch.int32 if a.dtype == torch.float32 else torch.int64)
    ib = b.view(torch.int32 if b.dtype == torch.float32 else torch.int64)
    return torch.equal(ia[~nan], ib[~nan])


def test_narrow_random_bit_patterns():
    rng = np.random.default_rng(1)
    u = rng.integers(0, 2**63, 4_000_000, dtype=np.int64) * rng.choice([1, -1], 4_000_000)
    x = torch.from_numpy(u).cuda().view(torch.float64)
    assert same_bits(narrow(x), x.to(torch.float32))


def test_narrow_near_binary32_range_and_ties():
    rng = np.random.default_rng(2)
    n = 4_000_000
    e = rng.integers(850, 1160, n, dtype=np.int64)  # binary32 subnormals .. overflow
    m = rng.integers(0, 2**52, n, dtype=np.int64)
    tie = rng.random(n) < 0.3
    m[tie] = (m[tie] & ~np.int64(0x1FFFFFFF)) | np.int64(0x10000000)  # exactly halfway between binary32 neighbours
    s = rng.integers(0, 2, n, dtype=np.int64) << np.int64(63)
    bits = s | (e << np.int64(52)) | m
    x = torch.from_numpy(bits).cuda().view(torch.float64)
    assert same_bits(narrow(x), x.to(torch.float32))


def test_narrow_special_values():
    f32 = np.finfo(np.float32)
    vals = [0.0, -0.0, np.inf, -np.inf, np.nan, float(f32.max), float(f32.max) * (1 + 2**-25),
            float(f32.max) * (1 + 2**-24), float(f32.tiny), float(f32.smallest_subnormal),
            float(f32.smallest_subnormal) / 2, float(f32.smallest_subnormal) * 0.75, 5e-324, -5e-324, 1e-300,
            1e300, 1.0, 1.0 + 2**-24, 1.0 + 3 * 2**-24, -(1.0 + 2**-24)]
    x = torch.tensor(vals, dtype=torch.float64, device="cuda")
    assert same_bits(narrow(x), x.to(torch.float32))


def test_widen_all_exponents_and_subnormals():
    rng = np.random.default_rng(3)
    u = np.concatenate([rng.integers(0, 2**32, 4_000_000, dtype=np.int64),
                        np.arange(0, 2**23, 7, dtype=np.int64),               # positive subnormals
                        np.arange(0, 2**23, 7, dtype=np.int64) | 0x80000000,  # negative subnormals
                        np.array([0x7F800000, 0xFF800000, 0x7FC00000, 0x7F800001, 0x80000000], dtype=np.int64)])
    x = torch.from_numpy(u.astype(np.uint32).view(np.int32)).cuda().view(torch.float32)
    assert same_bits(widen(x), x.to(torch.float64))


def test_round_trip_and_errors():
    x = torch.randn(100_000, dtype=torch.float64, device="cuda")
    y = widen(narrow(x))
    assert torch.equal(y, x.to(torch.float32).to(torch.float64))
    L = _lib.load()
    assert L.amg_narrow_f64(None, None, 5, None) == _lib.AMG_ERR_ARG
    assert L.amg_widen_f32(None, None, -1, None) == _lib.AMG_ERR_ARG
    assert L.amg_narrow_f64(None, None, 0, None) == 0
