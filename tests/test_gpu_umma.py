"""The tensor-core (tcgen05) BF16 matrix product of the proposal network
against an FP64 product of the same BF16 operands: FP32 accumulation of K
exact BF16 products, so the error is bounded by K ulp(FP32) of the sum of
|products| (tested at 1e-5 of that sum).  Shapes cover ragged M, N, K,
tiles of one row or column, and transposed operands read through strides."""
import numpy as np
import pytest

from gpu_util import load_ppl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppl():
    return load_ppl()


@pytest.mark.parametrize("M,N,K,ta,tb", [(128, 64, 64, 0, 0), (1024, 256, 64, 0, 0),
                                         (1024, 256, 256, 0, 0), (1024, 48, 256, 0, 0),
                                         (48, 256, 1024, 1, 1), (256, 256, 1024, 1, 1),
                                         (256, 64, 1024, 1, 1), (1, 1, 1, 0, 0),
                                         (77, 91, 33, 0, 1), (300, 130, 200, 1, 0)])
def test_umma_gemm_matches_fp64(ppl, M, N, K, ta, tb):
    import torch
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    a = torch.randn(M, K, generator=g).to(torch.bfloat16)
    b = torch.randn(N, K, generator=g).to(torch.bfloat16)
    # store transposed when asked, and read back through strides
    ad = (a.t().contiguous() if ta else a).cuda()
    bd = (b.t().contiguous() if tb else b).cuda()
    sam, sak = (1, M) if ta else (K, 1)
    sbn, sbk = (1, N) if tb else (K, 1)
    C, ws = ppl.ppl_gemm_bf16(ad, bd, M, N, K, sam, sak, sbn, sbk)
    torch.cuda.synchronize()
    assert ppl.ppl_workspace_status(ws) == 0
    ref = a.double() @ b.double().t()
    mag = a.double().abs() @ b.double().abs().t()
    err = (C.cpu().double() - ref).abs()
    assert torch.all(err <= 1e-5 * mag + 1e-30), float((err / (mag + 1e-30)).max())
