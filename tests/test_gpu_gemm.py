"""The tcgen05 BF16 GEMM (TMA + TMEM) against a reference FP32 matmul of the same
bf16 operands."""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [  # (M, N, K, bn)
    (128, 128, 64, 128), (128, 64, 64, 64), (300, 200, 160, 128), (4096, 1600, 16, 128),
    (1000, 800, 1600, 128), (16, 400, 4096, 128), (257, 16, 400, 64), (777, 512, 200, 256),
    # persistent kernel, double-buffered accumulator: several tiles per CTA, ragged edges
    (128, 160, 64, -160), (3000, 800, 1600, -160), (5000, 1600, 16, -160), (2049, 400, 800, -208),
    (4096, 512, 256, -256), (999, 384, 72, -128), (40000, 800, 1600, -160),
]


def _gemm(A, B, bn):
    from paper_2210_07094_gb300 import _lib
    M, K = A.shape
    N = B.shape[0]
    Cm = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.check(_lib.load().df_probe_gemm_bf16(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                                              C.c_void_p(Cm.data_ptr()), M, N, K, bn,
                                              C.c_void_p(err.data_ptr()),
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream)),
               "df_probe_gemm_bf16")
    torch.cuda.synchronize()
    return Cm, int(err.item())


@pytest.mark.parametrize("M,N,K,bn", SHAPES)
def test_gemm_matches_reference(M, N, K, bn):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    Cm, err = _gemm(A, B, bn)
    assert err == 0
    ref = A.double() @ B.double().T
    scale = (A.double().abs() @ B.double().abs().T)
    assert torch.all(torch.abs(Cm.double() - ref) <= 1e-5 * scale + 1e-6)
