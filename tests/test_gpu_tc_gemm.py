"""The tcgen05 tensor-core GEMM against a float64 product of the same bf16 values (the plain
reference), on shapes with ragged edges in M, N and K."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (512, 256, 784), (100, 200, 72), (256, 784, 512), (7, 9, 16),
                                   (129, 257, 65), (300, 520, 200), (1024, 1024, 1024)])
def test_bf16_gemm_matches_float64_reference(M, N, K):
    from paper_2602_19775_gb300 import ssa
    g = torch.Generator(device="cuda").manual_seed(M * 1000 + N + K)
    A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    D = ssa.bf16_gemm(A, B, bias)
    ref = A.double() @ B.double().T + bias.double()
    # binary32 accumulation of K exact products: |error| <= K u sum |a b|
    bound = K * 2.0 ** -24 * (A.double().abs() @ B.double().abs().T) + 1e-6
    assert torch.all((D.double() - ref).abs() <= bound), float((D.double() - ref).abs().max())


def test_bf16_gemm_integer_inputs_are_exact():
    from paper_2602_19775_gb300 import ssa
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randint(0, 256, (256, 784), device="cuda", generator=g).to(torch.bfloat16)   # counts 0..255
    B = torch.randint(-40, 41, (64, 784), device="cuda", generator=g).to(torch.bfloat16)   # small integers
    D = ssa.bf16_gemm(A, B)
    ref = A.double() @ B.double().T   # |sum| < 2^24: exact in binary32
    assert torch.equal(D.double(), ref)
