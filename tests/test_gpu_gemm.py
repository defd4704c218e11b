"""The tcgen05 BF16 GEMM of the learned warm start against an FP64 CPU
product of the same BF16 operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (256, 256, 256), (384, 64, 128),
                                   (128, 48, 192), (512, 128, 64)])
@pytest.mark.parametrize("relu,out_f32", [(False, True), (True, False)])
def test_gemm_matches_fp64_reference(M, N, K, relu, out_f32):
    import torch
    from paper_2311_18126_gb300 import ensure_built, gemm_bf16
    ensure_built()
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = (torch.randn(N, K, generator=g) / K ** 0.5).to(torch.bfloat16)
    bias = torch.randn(N, generator=g, dtype=torch.float32)
    ref = A.double() @ B.double().T + bias.double()
    if relu:
        ref = ref.clamp_min(0.0)
    C = torch.empty(M, N, dtype=torch.float32 if out_f32 else torch.bfloat16, device="cuda")
    gemm_bf16(A.cuda(), B.cuda(), bias.cuda(), C, relu=relu)
    out = C.double().cpu()
    if out_f32:
        tol = 1e-5 * (A.double().abs() @ B.double().abs().T + 1.0)
    else:
        tol = 2.0 ** -8 * ref.abs() + 1e-5 * (A.double().abs() @ B.double().abs().T + 1.0)
    assert torch.all((out - ref).abs() <= tol), float(((out - ref).abs() - tol).max())
