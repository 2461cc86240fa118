"""The library's table-driven exp and log against CUDA's and the host libm, and
the FP64 chain probe."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ulp_err(a, b):
    return np.abs(a - b) / np.spacing(np.abs(b))


@pytest.mark.parametrize("bits", [6, 8])
def test_exp_tang_within_two_ulp(bits):
    """Both tables (64 entries with the degree-5 polynomial, 256 with degree
    4): within 2 ulp of the host libm and of CUDA's exp."""
    from paper_2210_07094_gb300 import _lib
    L = _lib.load()
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-699.9, 699.9, 1 << 20), rng.uniform(-2, 2, 1 << 18),
                        rng.uniform(-1e-6, 1e-6, 1 << 12),
                        [0.0, -0.0, 1.0, -1.0, 699.0, -699.0, 700.0, -700.0, 709.0, -745.0, 1e-300]])
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    _lib.check(L.df_probe_exp(C.c_void_p(xd.data_ptr()), C.c_void_p(yd.data_ptr()), x.size, bits,
                              C.c_void_p(torch.cuda.current_stream().cuda_stream)), "df_probe_exp")
    y = yd.cpu().numpy()
    y_cuda = torch.exp(xd).cpu().numpy()
    y_host = np.exp(x)
    ok = y_host > 0
    assert np.max(_ulp_err(y[ok], y_host[ok])) <= 2.0
    assert np.max(_ulp_err(y[ok], y_cuda[ok])) <= 2.0
    assert y[x.size - 11] == 1.0 and y[x.size - 10] == 1.0


def test_log_tab_absolute_accuracy():
    """The table-driven logarithm of the rate kernels: within 2 ulp of
    max(1, |ln x|) of the exact value (ln T and the Troe log10s enter the rates
    as addends), on random magnitudes, near 1 and at the special values that go
    to the library log."""
    from paper_2210_07094_gb300 import _lib
    L = _lib.load()
    rng = np.random.default_rng(1)
    x = np.concatenate([10.0 ** rng.uniform(-307, 307, 1 << 20), rng.uniform(0.5, 2.0, 1 << 18),
                        1.0 + rng.uniform(-1e-6, 1e-6, 1 << 12), rng.uniform(200.0, 5000.0, 1 << 16),
                        [1.0, 2.0, 0.5, 300.0, 3000.0, 5e-324, 0.0, np.inf]])
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    _lib.check(L.df_probe_log(C.c_void_p(xd.data_ptr()), C.c_void_p(yd.data_ptr()), x.size,
                              C.c_void_p(torch.cuda.current_stream().cuda_stream)), "df_probe_log")
    y = yd.cpu().numpy()
    y_cuda = torch.log(xd).cpu().numpy()
    fin = np.isfinite(y_cuda)
    scale = np.maximum(1.0, np.abs(y_cuda[fin]))
    assert np.max(np.abs(y[fin] - y_cuda[fin]) / scale) <= 2 * 2.0 ** -52
    assert y[x.size - 1] == np.inf and y[x.size - 2] == -np.inf


def test_fp64_chain_probe():
    """df_probe_fp64_chains: rejects bad arguments; more warps and more
    independent chains never lower the FP64 throughput it reports."""
    import ctypes as C
    from paper_2210_07094_gb300 import _lib
    L = _lib.load()
    ns, gf = C.c_double(), C.c_double()
    assert L.df_probe_fp64_chains(0, 1, 100, C.byref(ns), C.byref(gf)) == -1
    assert L.df_probe_fp64_chains(1, 3, 100, C.byref(ns), C.byref(gf)) == -1
    assert L.df_probe_fp64_chains(1, 1, 0, C.byref(ns), C.byref(gf)) == -1
    res = {}
    for warps, chains in ((1, 1), (4, 1), (4, 8), (8, 8)):
        _lib.check(L.df_probe_fp64_chains(warps, chains, 2000, C.byref(ns), C.byref(gf)), "df_probe_fp64_chains")
        assert ns.value > 0 and gf.value > 0
        res[(warps, chains)] = gf.value
    assert res[(4, 1)] >= 0.9 * res[(1, 1)]
    assert res[(4, 8)] >= 0.9 * res[(4, 1)]
    assert res[(8, 8)] >= 0.9 * res[(4, 8)]
