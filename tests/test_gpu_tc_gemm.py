"""The BF16 tensor-core GEMM (tcgen05, TMA, TMEM) against a plain PyTorch
FP32 reference of the same op on the same BF16-rounded operands.

Products of two BF16 numbers are exact in FP32, so the only difference is the
FP32 accumulation order: |dY| <= 1e-5 sum_k |x_k w_k| + 1e-6.
"""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()


@pytest.mark.parametrize("rows,K,n,period", [(128, 128, 128, 1), (1000, 384, 128, 44), (777, 128, 112, 3),
                                             (300001, 384, 128, 44), (5, 64, 16, 1)])
def test_tc_gemm_matches_fp32_reference(rows, K, n, period):
    from paper_2307_14123_gb300.binding import test_gemm_bf16
    g = torch.Generator(device="cuda").manual_seed(rows + K)
    X = torch.randn(rows, K, device="cuda", generator=g).to(torch.bfloat16)
    W = (torch.randn(n, K, device="cuda", generator=g) / K ** 0.5).to(torch.bfloat16)
    bias = torch.randn(n, device="cuda", generator=g)
    Y, st = test_gemm_bf16(X, W, bias, period)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Xd, Wd = X.double(), W.double()
    ref = Xd @ Wd.T
    rb = torch.arange(rows, device="cuda") % period == 0
    ref[rb] += bias.double()
    scale = Xd.abs() @ Wd.abs().T
    err = (Y.double() - ref).abs()
    assert torch.all(err <= 1e-5 * scale + 1e-6), float((err / (scale + 1e-30)).max())
