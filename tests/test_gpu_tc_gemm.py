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


@pytest.mark.parametrize("rows,K,n,period", [(128, 128, 128, 1), (1000, 768, 256, 44), (777, 64, 112, 3),
                                             (200003, 256, 256, 44), (5, 32, 16, 1)])
def test_tf32x3_gemm_matches_fp64_reference(rows, K, n, period):
    """3 x TF32 split: the dropped x_lo w_lo term and the rounding of the low
    parts are each below 2^-22 |x||w|; with FP32 accumulation over K terms the
    bound 4e-6 sum_k |x_k w_k| (about 30 FP32 ulps) leaves room for the
    accumulation order while failing a missing cross term (about 2^-12)."""
    from paper_2307_14123_gb300.binding import test_gemm_tf32x3
    g = torch.Generator(device="cuda").manual_seed(7 * rows + K)
    X = torch.randn(rows, K, device="cuda", generator=g)
    W = torch.randn(n, K, device="cuda", generator=g) / K ** 0.5
    bias = torch.randn(n, device="cuda", generator=g)
    Y, st = test_gemm_tf32x3(X, W, bias, period)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Xd, Wd = X.double(), W.double()
    ref = Xd @ Wd.T
    rb = torch.arange(rows, device="cuda") % period == 0
    ref[rb] += bias.double()
    scale = Xd.abs() @ Wd.abs().T + rb[:, None].double() * bias.double().abs()
    err = (Y.double() - ref).abs()
    rel = float((err / (scale + 1e-30)).max())
    print(f"tf32x3 rows={rows} K={K} n={n}: max |dY|/sum|xw| {rel:.3e}")
    assert torch.all(err <= 4e-6 * scale + 1e-7), rel
