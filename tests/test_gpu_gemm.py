"""Tensor-core BF16 GEMM (tcgen05) against a float32 matmul of the same bf16 operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (200, 96, 128), (1000, 64, 576), (37, 5, 64)])
def test_gemm_matches_matmul(torch, M, N, K):
    from paper_2412_03451_gb300 import binding as B
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N)
    A = torch.randn(M, K, device="cuda", generator=g).bfloat16()
    Bm = torch.randn(N, K, device="cuda", generator=g).bfloat16()
    bias = torch.randn(N, device="cuda", generator=g)
    ref = A.float() @ Bm.float().T
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = torch.full((M, N), 7.0, device="cuda")
    B.ps_gemm_bf16(A, Bm, None, C, None, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert torch.allclose(C, ref, rtol=1e-4, atol=1e-3 * K ** 0.5), (C - ref).abs().max().item()
    # bias + ReLU, bf16 output, and accumulation into fp32
    C16 = torch.zeros(M, N, device="cuda", dtype=torch.bfloat16)
    B.ps_gemm_bf16(A, Bm, bias, None, C16, relu=True, err=err)
    C2 = ref.clone()
    B.ps_gemm_bf16(A, Bm, None, C2, None, accumulate=True, err=err)
    torch.cuda.synchronize()
    assert torch.allclose(C16.float(), torch.relu(ref + bias), rtol=1e-2, atol=1e-2 * K ** 0.5)
    assert torch.allclose(C2, 2 * ref, rtol=1e-4, atol=2e-3 * K ** 0.5)
    assert int(err.item()) == 0


def test_bounded_wait_times_out_and_context_stays_usable(torch):
    # a wait on an mbarrier that nothing arrives on (the GEMM's wait routine) gives up
    # after its poll limit and reports PS_ERR_TIMEOUT in the status word; no fault, and
    # the next GEMM on the same context is correct
    from paper_2412_03451_gb300 import binding as B
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.ps_wait_selftest(status, 1000)
    torch.cuda.synchronize()
    assert int(status.item()) == 1 << B.PS_ERR_TIMEOUT
    B.ps_wait_selftest(status, 1)
    torch.cuda.synchronize()
    assert int(status.item()) == 1 << B.PS_ERR_TIMEOUT
    A = torch.randn(256, 64, device="cuda").bfloat16()
    Bm = torch.randn(64, 64, device="cuda").bfloat16()
    C = torch.empty(256, 64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.ps_gemm_bf16(A, Bm, None, C, None, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert torch.allclose(C, A.float() @ Bm.float().T, rtol=1e-4, atol=8e-3)
