"""The tensor-core operand conventions the fused kernels rely on.

One 128 x n x k BF16 product per case through dp_selftest_mma (tcgen05.mma,
FP32 accumulation), operands in K-major or MN-major core-matrix layout, against
an FP64 host product of the same BF16-representable inputs.  The error bound is
FP32 accumulation over k <= 128 terms of magnitude ~1.
"""
import numpy as np
import pytest
import torch

import paper_2602_02234_b300 as dp

pytestmark = pytest.mark.gpu


def bf16(x):
    return torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).float().numpy()


@pytest.mark.parametrize("n,k", [(16, 16), (32, 128), (64, 32), (128, 64), (192, 48), (240, 112),
                                 (256, 128)])
@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_tcgen05_product(n, k, a_mn, b_mn):
    rng = np.random.default_rng(n * 1000 + k)
    A = bf16(rng.normal(size=(128, k)))
    B = bf16(rng.normal(size=(n, k)))
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    try:
        D = dp.selftest_mma(A, B, a_mn, b_mn, swap=0)
    except dp.DPError as e:
        assert e.code == dp.DP_ERR_ARG      # shapes the self-test cannot stage safely
        pytest.skip("shape not stageable in the self-test buffers")
    assert np.max(np.abs(D - ref)) <= 1e-5 * k


def test_bounded_wait_reports_timeout_and_context_survives():
    """A wait that nothing completes gives DP_ERR_TIMEOUT (no trap, no hang);
    the device stays usable afterwards."""
    assert dp.lib().dp_selftest_timeout(4096) == dp.DP_ERR_TIMEOUT
    A = bf16(np.ones((128, 16)))
    B = bf16(np.ones((16, 16)))
    assert np.allclose(dp.selftest_mma(A, B), 16.0)


def test_product_rate_self_test():
    """dp_selftest_mma_rate: a 128 x n x 16 product costs at least the
    tensor-core time of its n columns, and wider products never cost less
    than narrower ones (one or four issuing threads)."""
    r16 = dp.selftest_mma_rate(16)
    r32 = dp.selftest_mma_rate(32)
    r128 = dp.selftest_mma_rate(128)
    r32x4 = dp.selftest_mma_rate(32, issuers=4)
    for r in (r16, r32, r128, r32x4):
        assert np.isfinite(r) and r > 0
    assert r128 >= r16
    # 128 x 128 x 16 is 2^18 multiply-adds; no SM does more than 8,192 per cycle
    assert r128 >= 32.0
    with pytest.raises(dp.DPError):
        dp.selftest_mma_rate(24)
