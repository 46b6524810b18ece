"""GPU tests of the learned surrogate's tensor-core path: the BF16 tcgen05 GEMM against
an FP32 product of the same BF16 operands, then (below) the network against the FP64
surrogate oracle (oracle/mlp.py)."""
import numpy as np
import pytest
import torch

from paper_2209_13775_gb300 import lcs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    c = lcs.lcs_create(0, torch.cuda.current_stream())
    yield c
    lcs.lcs_destroy(c)


@pytest.mark.parametrize("M,N,K,splits", [(128, 128, 16, 1), (256, 128, 64, 1), (384, 256, 208, 1),
                                          (128, 16, 128, 1), (300, 128, 144, 1), (128, 128, 4096, 8),
                                          (1024, 16, 1024, 3)])
def test_gemm_bf16_matches_fp32_product(ctx, M, N, K, splits):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    want = A.double() @ B.double().T
    Ad, Bd = A.cuda(), B.cuda()
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    if splits > 1:
        C.zero_()
    lcs.lcs_gemm_bf16(ctx, Ad, Bd, C, splits=splits)
    lcs.lcs_synchronize(ctx)
    got = C.cpu().double()
    # FP32 accumulation of exact BF16 products: error ~ K * 2^-24 * sum |a b|
    bound = (A.double().abs() @ B.double().abs().T) * (K * 2.0 ** -23) + 1e-6
    assert torch.isfinite(got).all()
    assert ((got - want).abs() <= bound).all(), float((got - want).abs().max())
    # accumulate mode adds onto C
    lcs.lcs_gemm_bf16(ctx, Ad, Bd, C, splits=1, accumulate=True)
    lcs.lcs_synchronize(ctx)
    assert ((C.cpu().double() - 2 * want).abs() <= 2 * bound).all()
