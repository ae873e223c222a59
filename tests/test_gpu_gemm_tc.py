"""The BF16 tensor-core GEMM (tcgen05, FP32 accumulate in tensor memory) used
by the learned warm start, against an FP32 CPU product of the same bf16
values.  Bf16 x bf16 products are exact in FP32; only the summation order
differs, so the bound is a few FP32 ulps of sum |a||b|."""
import pytest
import torch

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (16, 64), (64, 16), (64, 64), (64, 128), (128, 64)]


@pytest.fixture(scope="module")
def ctx():
    from paper_1903_12359_gb300 import build
    build.build()
    from paper_1903_12359_gb300 import api
    return api.Context()


def _ref(A, Bt):
    return A.float().cpu() @ Bt.float().cpu().T


@pytest.mark.parametrize("N,K", SHAPES)
@pytest.mark.parametrize("M", [1, 128, 1000, 4099])
def test_gemm_store_f32(ctx, N, K, M):
    g = torch.Generator().manual_seed(N * 1000 + K + M)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    Bt = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = ctx.selftest_gemm_bf16(A, Bt, epilogue=0).cpu()
    R = _ref(A, Bt)
    bound = 4 * K * 2.0 ** -24 * (A.float().abs().cpu() @ Bt.float().abs().cpu().T) + 1e-30
    assert torch.all((C - R).abs() <= bound), float(((C - R).abs() / bound).max())


@pytest.mark.parametrize("N,K", [(64, 64), (64, 128), (16, 64)])
def test_gemm_bias_relu_bf16_and_bias_f32(ctx, N, K):
    M = 777
    g = torch.Generator().manual_seed(7)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    Bt = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    b = torch.randn(N, generator=g).float().cuda()
    R = _ref(A, Bt) + b.cpu()
    C2 = ctx.selftest_gemm_bf16(A, Bt, epilogue=2, bias=b).cpu()
    assert torch.allclose(C2, R, rtol=1e-5, atol=1e-4)
    C1 = ctx.selftest_gemm_bf16(A, Bt, epilogue=1, bias=b).cpu()
    assert C1.dtype == torch.bfloat16
    assert torch.equal(C1, torch.relu(C2).to(torch.bfloat16))


def test_gemm_rejects_unsupported_shapes(ctx):
    from paper_1903_12359_gb300 import api
    A = torch.zeros(128, 48, dtype=torch.bfloat16, device="cuda")
    Bt = torch.zeros(64, 48, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(api.PgcpError) as e:
        ctx.selftest_gemm_bf16(A, Bt)
    assert e.value.code == "ARG"
