"""The GELU of the GEMM epilogues (Sec. 2.3's activation, z Phi(z)) and its
derivative against the exact function in FP64 on a dense grid."""
import ctypes as C

import numpy as np
import pytest
from scipy.special import erfc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(x, derivative):
    from paper_2210_07094_gb300 import _lib
    L = _lib.load()
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.empty_like(xd)
    _lib.check(L.df_probe_gelu(C.c_void_p(xd.data_ptr()), C.c_void_p(yd.data_ptr()), x.size, derivative,
                               C.c_void_p(torch.cuda.current_stream().cuda_stream)), "df_probe_gelu")
    return yd.cpu().numpy().astype(np.float64)


def _grid():
    rng = np.random.default_rng(3)
    x = np.concatenate([np.linspace(-13.0, 13.0, 1 << 20), rng.normal(0.0, 2.0, 1 << 18),
                        rng.uniform(-1e-3, 1e-3, 1 << 12), [0.0, -0.0, 1e-30, -1e-30, 40.0, -40.0]])
    return x.astype(np.float32).astype(np.float64)


def test_gelu_relative_error():
    x = _grid()
    y = _run(x, 0)
    exact = 0.5 * x * erfc(-x / np.sqrt(2.0))  # erfc keeps the negative tail exact
    tiny = np.abs(exact) < 1e-35  # below the FP32 range: the value flushes to (-)0
    rel = np.abs(y - exact)[~tiny] / np.abs(exact[~tiny])
    # the exp2 argument (-a^2 + P(t)) log2(e) carries one FP32 rounding of its
    # size: relative error grows with x^2 in the far negative tail
    bound = np.where(np.abs(x[~tiny]) <= 8.0, 1e-5, 5e-5)
    assert np.all(rel <= bound), (rel.max(), x[~tiny][np.argmax(rel / bound)])
    assert np.all(np.abs(y[tiny]) <= 1e-35)
    # after the BF16 rounding the epilogue applies, almost every value is the
    # correctly rounded one (a flip needs the value within the FP32 error,
    # ~3e-7 relative in the body, of a BF16 rounding boundary)
    b = lambda a: torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).float().numpy()  # noqa: E731
    flips = float(np.mean(b(y) != b(exact)))
    print({"bf16_flip_rate": flips, "max_rel": float(rel.max())})
    assert flips < 5e-4


def test_gelu_derivative_error():
    x = _grid()
    y = _run(x, 1)
    exact = 0.5 * erfc(-x / np.sqrt(2.0)) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)
    # Phi(z) and z phi(z) cancel near z = -0.75: an absolute floor of a few FP32
    # roundings of terms of size 0.2
    assert np.all(np.abs(y - exact) <= 2e-5 * np.abs(exact) + 1e-6)
