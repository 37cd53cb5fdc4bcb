"""The tcgen05 BF16 GEMM (mgmc_tc_gemm) against an FP64 matmul of the same BF16 values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    from paper_2407_12149_gb300 import build
    build.build()
    return torch


def _ref(torch, A, B):
    return A.double().cpu().numpy() @ B.double().cpu().numpy().T


@pytest.mark.parametrize("M,N,K,splits", [(128, 32, 64, 1), (256, 64, 128, 1), (384, 128, 192, 1),
                                          (128, 256, 64, 1), (200, 40, 72, 1), (1000, 96, 296, 1),
                                          (256, 64, 4096, 4), (320, 8, 27 * 8, 3)])
def test_tc_gemm_matches_fp64(torch_mod, M, N, K, splits):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import tc_gemm
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    lda = (K + 7) // 8 * 8
    Ab = torch.zeros(M, lda, dtype=torch.bfloat16, device="cuda")
    Bb = torch.zeros(N, lda, dtype=torch.bfloat16, device="cuda")
    Ab[:, :K] = torch.randn(M, K, generator=g, device="cuda").bfloat16()
    Bb[:, :K] = torch.randn(N, K, generator=g, device="cuda").bfloat16()
    C = tc_gemm(Ab[:, :K], Bb[:, :K], splits=splits)
    torch.cuda.synchronize()
    ref = _ref(torch, Ab[:, :K], Bb[:, :K])
    err = np.abs(C.cpu().numpy() - ref).max()
    # FP32 accumulation of K products of BF16 values (|a b| <~ 10): rounding ~ K * 2^-24 * 10
    assert err <= 1e-5 * K + 1e-5, err


def test_tc_gemm_epilogue_bias_relu_bf16(torch_mod):
    torch = torch_mod
    from paper_2407_12149_gb300.mgmc import tc_gemm, EPI_BIAS, EPI_RELU, EPI_BF16
    g = torch.Generator(device="cuda").manual_seed(5)
    M, N, K = 512, 64, 288
    A = torch.randn(M, K, generator=g, device="cuda").bfloat16()
    B = torch.randn(N, K, generator=g, device="cuda").bfloat16()
    bias = torch.randn(N, generator=g, device="cuda")
    C = tc_gemm(A, B, epilogue=EPI_BIAS | EPI_RELU | EPI_BF16, bias=bias)
    torch.cuda.synchronize()
    ref = np.maximum(_ref(torch, A, B) + bias.double().cpu().numpy()[None, :], 0.0)
    got = C.float().cpu().numpy()
    # BF16 output rounding: relative 2^-8
    assert np.all(np.abs(got - ref) <= 2 ** -8 * np.abs(ref) + 1e-3)
