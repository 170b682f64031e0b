"""The tcgen05 tensor-core GEMM against a float64 product of the same bf16 values (the plain
reference), on shapes with ragged edges in M, N and K, with and without the split-K work buffer."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("split_k", [False, True])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (512, 256, 784), (100, 200, 72), (256, 784, 512), (7, 9, 16),
                                   (129, 257, 65), (300, 520, 200), (1024, 1024, 1024), (512, 256, 6272),
                                   (130, 250, 4104), (64, 64, 4096)])
def test_bf16_gemm_matches_float64_reference(M, N, K, split_k):
    from paper_2602_19775_gb300 import ssa
    g = torch.Generator(device="cuda").manual_seed(M * 1000 + N + K)
    A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    D = ssa.bf16_gemm(A, B, bias, split_k=split_k)
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


def test_split_k_is_taken_deterministic_and_checked():
    """The E1-shaped product (512 x 256, K = 6,272) has 4 output tiles, so the work buffer splits K; two calls
    give the same bits, the split and unsplit results agree to binary32 accumulation, a short buffer is
    refused, and K = 0 writes the bias."""
    from paper_2602_19775_gb300 import SSAError, ssa
    from paper_2602_19775_gb300 import _lib
    L = _lib.lib()
    M, N, K = 512, 256, 6272
    words = int(L.ssa_bf16_gemm_work_words(M, N, K))
    assert words >= 2 * M * N and words % (M * N) == 0
    assert int(L.ssa_bf16_gemm_work_words(8192, 8192, 8192)) == 0   # 2,048 tiles: no split
    assert int(L.ssa_bf16_gemm_work_words(512, 256, 192)) == 0      # three K blocks: no split
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    d1, d2 = ssa.bf16_gemm(A, B, split_k=True), ssa.bf16_gemm(A, B, split_k=True)
    assert torch.equal(d1, d2)
    d0 = ssa.bf16_gemm(A, B, split_k=False)
    bound = 2 * K * 2.0 ** -24 * (A.double().abs() @ B.double().abs().T)
    assert torch.all((d1.double() - d0.double()).abs() <= bound)
    D = torch.empty((M, N), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    work = torch.empty(words, dtype=torch.float64, device="cuda")
    with pytest.raises(SSAError):
        ssa.check(L.ssa_bf16_gemm(ssa._ptr(A), ssa._ptr(B), M, N, K, K, K, None, ssa._ptr(D), N, ssa._ptr(work),
                                  words - 1, ssa._ptr(err), ssa._stream()))
    bias = torch.randn(N, device="cuda", generator=g)
    e = ssa.bf16_gemm(A[:, :0], B[:, :0], bias)
    assert torch.equal(e, bias.expand(M, N))
