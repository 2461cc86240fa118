"""The library's table-driven exp against CUDA's exp and the host libm."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ulp_err(a, b):
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_exp_tang_within_two_ulp():
    from paper_2210_07094_gb300 import _lib
    L = _lib.load()
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-699.9, 699.9, 1 << 20), rng.uniform(-2, 2, 1 << 18),
                        rng.uniform(-1e-6, 1e-6, 1 << 12),
                        [0.0, -0.0, 1.0, -1.0, 699.0, -699.0, 700.0, -700.0, 709.0, -745.0, 1e-300]])
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    _lib.check(L.df_probe_exp(C.c_void_p(xd.data_ptr()), C.c_void_p(yd.data_ptr()), x.size,
                              C.c_void_p(torch.cuda.current_stream().cuda_stream)), "df_probe_exp")
    y = yd.cpu().numpy()
    y_cuda = torch.exp(xd).cpu().numpy()
    y_host = np.exp(x)
    ok = y_host > 0
    assert np.max(_ulp_err(y[ok], y_host[ok])) <= 2.0
    assert np.max(_ulp_err(y[ok], y_cuda[ok])) <= 2.0
    assert y[x.size - 11] == 1.0 and y[x.size - 10] == 1.0
