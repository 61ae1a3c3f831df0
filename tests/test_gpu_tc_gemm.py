"""tcgen05 tensor-core GEMM against a plain PyTorch FP64 product of the same FP32 operands.
The sizes cover each tile width the launcher picks (128, 144 and 160 columns) and ragged edges."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

afqmc = pytest.importorskip("paper_2506_09611_gb300.afqmc")
torch = pytest.importorskip("torch")


def _run(kind, M, N, K, c_trans=0, pad=8, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    lda = K + pad
    A = torch.zeros((M, lda), dtype=torch.float32)
    A[:, :K] = torch.randn((M, K), generator=g)
    Bt = torch.zeros((N, lda), dtype=torch.float32)
    Bt[:, :K] = torch.randn((N, K), generator=g)
    A, Bt = A.cuda(), Bt.cuda()
    ldc = (M if c_trans else N) + pad
    C = torch.full(((N if c_trans else M), ldc), float("nan"), dtype=torch.float32, device="cuda")
    afqmc.afqmc_debug_gemm(kind, M, N, K, A.data_ptr(), lda, Bt.data_ptr(), lda, C.data_ptr(), ldc, c_trans,
                           torch.cuda.current_stream())
    ref = A[:, :K].double() @ Bt[:, :K].double().T
    got = C[:, :M].double().T if c_trans else C[:, :N].double()
    assert torch.isnan(C[:, (M if c_trans else N):]).all()  # padding untouched
    return (torch.linalg.norm(got - ref) / torch.linalg.norm(ref)).item()


def _fp32_reference_error(M, N, K, seed=0):
    """Relative error of a plain FP32 product (TF32 disabled) of the same operands."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn((M, K), generator=g)
    B = torch.randn((N, K), generator=g)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        c32 = (A.cuda() @ B.cuda().T).double()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    ref = A.double().cuda() @ B.double().cuda().T
    return (torch.linalg.norm(c32 - ref) / torch.linalg.norm(ref)).item()


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (256, 128, 64), (200, 136, 72), (1600, 1600, 1600),
                                   (36, 36, 36), (130, 260, 100), (1152, 2304, 2304), (1500, 1590, 200)])
def test_tc_gemm_split3_is_fp32_accurate(M, N, K):
    """The three-term split stays within a small factor of a plain FP32 product's error."""
    err = _run(2, M, N, K)
    assert err < max(2e-6, 8 * _fp32_reference_error(M, N, K))


@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (300, 170, 96), (1600, 1600, 256), (1152, 2304, 128)])
def test_tc_gemm_tf32_one_pass(M, N, K):
    err = _run(1, M, N, K)
    assert 1e-5 < err < 3e-3  # TF32 inputs: ~1e-3 relative, clearly not FP32


def test_tc_gemm_transposed_output():
    assert _run(2, 300, 200, 160, c_trans=1) < 2e-6
    assert _run(2, 1152, 2304, 96, c_trans=1) < 2e-6  # 144-wide tiles (one wave of 144 on 152 SMs)
    assert _run(2, 1500, 1590, 64, c_trans=1) < 2e-6  # 160-wide tiles, ragged in both dimensions
