"""The measured FP64 FMA rate (dg_fp64_fma_rate), the denominator beside the nominal 1.25 TFLOP/s
(2 FMA lanes x 152 SMs x 2.07 GHz x 2 flops) of the FP64-bound kernels: positive, and not above the
nominal rate by more than clock and counting slack."""

import pytest

from tests._gpu import torch_cuda

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_plausible():
    torch_cuda()
    from paper_2512_17101_gb300 import dg
    r = dg.dg_fp64_fma_rate()
    print(f"measured FP64 FMA rate {r:.3f} TFLOP/s")
    assert 0.2 < r < 1.25 * 1.1
