"""The tcgen05 BF16 GEMM (C = A B^T + bias, ReLU, mask) against a plain FP32
matmul of the same BF16 inputs (CPU)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2007_12273_gb300 import build, gm as gm_
    build.build()
    gm_.load()
    return gm_


@pytest.mark.parametrize("M,N,K", [(128, 32, 64), (128, 256, 64), (256, 256, 576), (300, 112, 130),
                                   (1000, 300, 256), (64, 16, 8)])
def test_gemm_matches_fp32_reference(gm, M, N, K):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g)
    ref = A.float() @ B.float().T + bias
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    # operands in row-padded storage (leading dimension a multiple of 8)
    Kp = (K + 7) // 8 * 8
    Ad = torch.zeros(M, Kp, dtype=torch.bfloat16, device="cuda")
    Bd = torch.zeros(N, Kp, dtype=torch.bfloat16, device="cuda")
    Ad[:, :K] = A.cuda()
    Bd[:, :K] = B.cuda()
    C = gm.gm_gemm_bf16(Ad[:, :K], Bd[:, :K], bias=bias.cuda(), err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    torch.testing.assert_close(C.cpu(), ref, rtol=1e-4, atol=1e-3 * K ** 0.5)


def test_gemm_relu_mask_and_bf16_output(gm):
    g = torch.Generator().manual_seed(1)
    M, N, K = 256, 128, 192
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    mask = (torch.rand(M, N, generator=g) > 0.5).to(torch.bfloat16)
    ref = torch.relu(A.float() @ B.float().T) * (mask.float() > 0)
    outb = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    C = gm.gm_gemm_bf16(A.cuda(), B.cuda(), relu=True, mask=mask.cuda(), out_bf16=outb)
    torch.cuda.synchronize()
    torch.testing.assert_close(C.float().cpu(), ref.to(torch.bfloat16).float(), rtol=1e-2, atol=1e-2)


@pytest.mark.parametrize("ld", [304, 301])
def test_gemm_epilogue_vector_and_element_paths(gm, ld):
    """Output rows padded to a 16-byte multiple take the epilogue's vector
    stores for every full 16-column chunk (the last, ragged chunk of N = 300
    element by element); an odd leading dimension takes the element path
    throughout.  Both must write the same values and nothing outside the
    N columns of each row."""
    g = torch.Generator().manual_seed(ld)
    M, N, K = 200, 300, 96
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g)
    mask = (torch.rand(M, ld, generator=g) > 0.3).to(torch.bfloat16)
    ref = torch.relu(A.float() @ B.float().T + bias) * (mask[:, :N].float() > 0)
    big = torch.full((M, ld), 7.0, dtype=torch.float32, device="cuda")
    out = big[:, :N]
    C = gm.gm_gemm_bf16(A.cuda(), B.cuda(), bias=bias.cuda(), relu=True, mask=mask.cuda()[:, :N],
                        out_f32=out)
    torch.cuda.synchronize()
    torch.testing.assert_close(C.cpu(), ref, rtol=1e-4, atol=1e-3 * K ** 0.5)
    assert torch.all(big[:, N:].cpu() == 7.0)
    bigb = torch.full((M, ld), 7.0, dtype=torch.bfloat16, device="cuda")
    Cb = gm.gm_gemm_bf16(A.cuda(), B.cuda(), bias=bias.cuda(), relu=True, mask=mask.cuda()[:, :N],
                         out_bf16=bigb[:, :N])
    torch.cuda.synchronize()
    torch.testing.assert_close(Cb.float().cpu(), ref.to(torch.bfloat16).float(), rtol=1e-2, atol=1e-2)
    assert torch.all(bigb[:, N:].float().cpu() == 7.0)
