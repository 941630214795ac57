"""The tiled tensor-core GEMM (letkf_gemm_selftest) against an FP64 product: C = A B^T for FP32
A (M x K) and B (N x K), ragged and tile-aligned shapes, both CTA tile widths, B read K-major or
(given as K x N) MN-major, single BF16 and the three-product split.  Bound per element, from the arithmetic: the operands' representation error
(2^-9 per BF16 operand; 3 x 2^-17 for the split) plus FP32 accumulation over K terms (K 2^-24),
times sum_k |A_ik| |B_jk|."""

import numpy as np
import pytest
import torch

from paper_1310_5954_gb300 import _lib
from paper_1310_5954_gb300 import build as builder

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    builder.build()
    _lib.load()


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (200, 130, 100), (1, 1, 1), (300, 257, 1000),
                                   (1025, 1025, 9264), (2048, 1024, 1024), (1024, 1024, 1024)])
@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("bn,b_mn", [(64, 0), (128, 0), (256, 0), (64, 1)])
def test_gemm_matches_fp64(M, N, K, split, bn, b_mn):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = (rng.standard_normal((N, K)) * 2.0 + 0.5).astype(np.float32)
    a = torch.as_tensor(A, device="cuda")
    # b_mn: B handed over as its transpose (K x N) and read MN-major, C = A (B^T)
    b = torch.as_tensor(np.ascontiguousarray(B.T) if b_mn else B, device="cuda")
    c = torch.full((M, N), np.nan, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = _lib.load().letkf_gemm_selftest(a.data_ptr(), b.data_ptr(), c.data_ptr(), M, N, K, split, bn, b_mn, st)
    assert rc == 0
    C = c.cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    eps = (3 * 2.0 ** -17 if split else 2 * 2.0 ** -9) + K * 2.0 ** -24
    err = np.abs(C - ref)
    assert np.isfinite(C).all()
    assert (err <= eps * scale + 1e-30).all(), float((err / (scale + 1e-30)).max())
    # the split is what makes FP32-level products
    if split and K >= 64:
        assert float((err / scale).max()) < 1e-4
