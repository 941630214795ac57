"""Tensor-core product of the fused path (tcgen05, BF16 operands, FP32 accumulation) vs float64.

Bound per element: BF16 keeps 8 significant bits (unit roundoff u = 2^-8), so with single
BF16 operands each product carries a relative error of at most 2u + u^2; with the high/low
split the dropped low*low term and the rounding of the low parts leave about 3u^2; FP32
accumulation adds k * 2^-24.  Both are checked against
|A| |B|^T, the natural scale of the sum.
"""

import pytest
import torch

from paper_1310_5954_gb300 import _lib
from paper_1310_5954_gb300 import build as builder

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


@pytest.mark.parametrize("n,k", [(16, 16), (112, 112), (48, 64), (256, 128), (128, 32), (32, 48)])
@pytest.mark.parametrize("terms", [1, 3])
@pytest.mark.parametrize("b_layout", [0, 1])
def test_umma_product(n, k, terms, b_layout):
    if b_layout == 1 and n > k:
        pytest.skip("MN-major operand checked on n <= k shapes (the fused path uses square ones)")
    g = torch.Generator(device="cpu").manual_seed(n * 1000 + k + terms + 7 * b_layout)
    A = torch.randn(128, k, generator=g, dtype=torch.float32)
    B = torch.randn(n, k, generator=g, dtype=torch.float32)
    A[:, 0] *= 100.0          # rows and columns of different scales
    B[3 % n] *= 1e-3
    Bin = B if b_layout == 0 else B.T.contiguous()     # layout 1 takes op(B) = B as a k x n matrix
    Ad, Bd = A.cuda(), Bin.cuda()
    D = torch.full((128, n), float("nan"), device="cuda")
    rc = _lib.letkf_umma_selftest(Ad.data_ptr(), Bd.data_ptr(), D.data_ptr(), n, k, terms, b_layout,
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    ref = A.double() @ B.double().T
    scale = A.double().abs() @ B.double().abs().T
    u = 2.0 ** -8
    bound = ((2 * u + u * u) if terms == 1 else 4 * u * u) * scale + 1e-6
    err = (D.cpu().double() - ref).abs()
    assert torch.isfinite(D).all()
    assert bool((err <= bound).all()), float((err / bound).max())


def test_umma_rejects_bad_shapes():
    assert _lib.letkf_umma_selftest(1, 1, 1, 20, 16, 1) == _lib.LETKF_EINVAL
    assert _lib.letkf_umma_selftest(1, 1, 1, 16, 144, 1) == _lib.LETKF_EINVAL
    assert _lib.letkf_umma_selftest(1, 1, 1, 16, 16, 2) == _lib.LETKF_EINVAL
    assert _lib.letkf_umma_selftest(1, 1, 1, 16, 16, 1, 2) == _lib.LETKF_EINVAL


def test_bounded_wait_gives_up_and_the_context_survives():
    """A device-side wait on a barrier nothing completes ends after its limit (~1 ms here) with
    LETKF_ETIMEOUT, not a hang; the context keeps working: the same wait with the arrival
    completes, and a filter step afterwards runs clean."""
    import time
    t0 = time.perf_counter()
    assert _lib.letkf_wait_selftest(2_000_000, 0) == _lib.LETKF_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert _lib.letkf_wait_selftest(2_000_000, 1) == _lib.LETKF_OK
    assert _lib.letkf_wait_selftest(10, 1) == _lib.LETKF_EINVAL
    from _gpu_common import gpu_filter, slopes
    y, _ = slopes("tiny-8x8", 2)
    f = gpu_filter("tiny-8x8", "mixed", "fused")
    f.step(torch.as_tensor(y[0], dtype=torch.float32, device="cuda"))
    assert f.sync() == 0
    f.close()
