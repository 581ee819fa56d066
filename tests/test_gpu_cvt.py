"""The integer-pipe FP64 <-> FP32 conversions of the mixed-precision kernels against the
hardware conversions (torch's .float() / .double() on the GPU): bit for bit."""

import numpy as np
import pytest

from tests._gpu import torch_cuda

pytestmark = pytest.mark.gpu


def _doubles():
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2**63, size=200_000, dtype=np.uint64)
    bits |= rng.integers(0, 2, size=bits.size, dtype=np.uint64) << np.uint64(63)
    x = bits.view(np.float64)
    # values in and around FP32's range, and the rounding boundaries of their last place
    y = rng.normal(size=100_000) * 10.0 ** rng.integers(-45, 40, size=100_000)
    f = rng.normal(size=50_000).astype(np.float32)
    ulp = np.spacing(f).astype(np.float64)
    ties = f.astype(np.float64) + 0.5 * ulp                       # exact halfway points
    near = f.astype(np.float64) + 0.5 * ulp * (1 + 2.0 ** -30)     # just above halfway
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 3.4028234663852886e38,
                     3.4028235677973366e38, 3.402823669209385e38, 1.1754943508222875e-38,
                     1.1754942106924411e-38, 1.401298464324817e-45, 7.006492321624085e-46, 5e-324,
                     2.2250738585072014e-308, 1.7976931348623157e308, 0.1, 1.0 / 3.0])
    return np.concatenate([x, y, ties, near, edge, -edge])


def test_round_to_float_matches_hardware():
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    x = torch.tensor(_doubles(), device="cuda")
    y = torch.empty(x.numel(), device="cuda", dtype=torch.float32)
    dg.dg_round_to_float(x, y)
    want = x.float()
    got_b, want_b = y.view(torch.int32), want.view(torch.int32)
    nan = torch.isnan(want)
    assert bool(torch.equal(torch.isnan(y), nan))
    assert bool(torch.equal(got_b[~nan], want_b[~nan]))


def test_widen_to_double_matches_hardware():
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    rng = np.random.default_rng(6)
    bits = rng.integers(0, 2**32, size=300_000, dtype=np.uint64).astype(np.uint32)
    f = np.concatenate([bits.view(np.float32),
                        np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, 3.4028235e38, 1.1754944e-38],
                                 dtype=np.float32)])
    x = torch.tensor(f, device="cuda")
    y = torch.empty(x.numel(), device="cuda", dtype=torch.float64)
    dg.dg_widen_to_double(x, y)
    want = x.double()
    sub = (x != 0) & (x.abs() < 1.1754943508222875e-38)  # float subnormals: flushed to signed zero
    nan = torch.isnan(want)
    assert bool(torch.equal(torch.isnan(y), nan))
    keep = ~nan & ~sub
    assert bool(torch.equal(y.view(torch.int64)[keep], want.view(torch.int64)[keep]))
    assert bool((y[sub] == 0).all()) and bool(torch.equal(torch.signbit(y[sub]), torch.signbit(x[sub])))


def test_split_to_float_pair_matches_fp64_residual():
    """hi = x rounded to FP32, lo = (x - hi) rounded to FP32, the residual taken in FP64."""
    torch = torch_cuda()
    from paper_2512_17101_gb300 import dg
    x = torch.tensor(_doubles(), device="cuda")
    keep = torch.isfinite(x) & (x.float().abs() < 3.0e38)
    x = x[keep].contiguous()
    hi = torch.empty(x.numel(), device="cuda", dtype=torch.float32)
    lo = torch.empty_like(hi)
    dg.dg_split_to_float_pair(x, hi, lo)
    want_hi = x.float()
    want_lo = (x - want_hi.double()).float()
    assert bool(torch.equal(hi.view(torch.int32), want_hi.view(torch.int32)))
    # signed zeros of the residual may differ; compare values
    bad = lo != want_lo
    assert not bool(bad.any()), (x[bad][:5].tolist(), lo[bad][:5].tolist(), want_lo[bad][:5].tolist())
