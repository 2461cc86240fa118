"""The adjoint entry point that allocates nothing (df_chem_adjoint_static).

It serves callers that cannot allocate device memory at the moment they need a
gradient (under an external memory pool, in a loop that forbids allocation).  The test calls it through the C ABI twice in a row,
on different inputs, and checks each result against df_chem_adjoint with a
caller-provided workspace; then checks that an oversize request is refused
with a clear error.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def test_static_scratch_adjoint_matches_workspace_adjoint():
    import paper_2210_07094_gb300 as df
    from paper_2210_07094_gb300 import _lib, synth

    L = _lib.load()
    mech = synth.h2_air_mechanism()
    m = df.Mechanism(mech)
    n, max_steps = 512, 16
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (41, 42):  # two calls in a row share the one scratch array
        f = synth.field(1, mech, n, seed=seed)
        T, p, Y = (torch.tensor(np.ascontiguousarray(f[k]), device=DEV) for k in ("T", "p", "Y"))
        rng = np.random.default_rng(seed)
        gT = torch.tensor(rng.standard_normal(n), device=DEV)
        gY = torch.tensor(rng.standard_normal((m.n_species, n)), device=DEV)
        gQ = torch.tensor(rng.standard_normal(n) * 1e-9, device=DEV)
        ref = df.adjoint(m, T, p, Y, f["dt"], gT, gY, gQ, max_steps=max_steps)
        gT0 = torch.full((n,), np.nan, dtype=torch.float64, device=DEV)
        gY0 = torch.full((m.n_species, n), np.nan, dtype=torch.float64, device=DEV)
        glnA = torch.full((m.n_reactions,), np.nan, dtype=torch.float64, device=DEV)
        status = torch.full((n,), -1, dtype=torch.int32, device=DEV)
        nsub = torch.full((n,), -1, dtype=torch.int32, device=DEV)
        rc = L.df_chem_adjoint_static(m.handle, n, _ptr(T), _ptr(p), _ptr(Y), C.c_double(f["dt"]), None,
                                      max_steps, _ptr(gT), _ptr(gY), _ptr(gQ), _ptr(gT0), _ptr(gY0), _ptr(glnA),
                                      _ptr(status), _ptr(nsub), stream)
        _lib.check(rc, "df_chem_adjoint_static")
        torch.cuda.synchronize()
        assert torch.equal(status, ref["status"]) and int(status.abs().sum()) == 0
        assert torch.equal(nsub, ref["nsub"])
        for a, b in ((gT0, ref["gT0"]), (gY0, ref["gY0"]), (glnA, ref["g_lnA"])):
            assert torch.allclose(a, b, rtol=1e-12, atol=0.0)


def test_static_scratch_adjoint_refuses_oversize_requests():
    import paper_2210_07094_gb300 as df
    from paper_2210_07094_gb300 import _lib, synth

    L = _lib.load()
    m = df.Mechanism(synth.h2_air_mechanism())
    one = torch.zeros(16, dtype=torch.float64, device=DEV)
    st = torch.zeros(16, dtype=torch.int32, device=DEV)
    rc = L.df_chem_adjoint_static(m.handle, 65536, _ptr(one), _ptr(one), _ptr(one), C.c_double(1e-6), None, 16,
                                  None, None, None, _ptr(one), _ptr(one), _ptr(one), _ptr(st), None, None)
    assert rc == -5  # DF_EWORKSPACE
    buf = C.create_string_buffer(512)
    L.df_get_last_error_detail(buf, 512)
    assert b"4 MiB" in buf.value


def test_static_scratch_adjoint_rejects_wrapping_sizes_and_host_pointers():
    """Sizes whose checkpoint count overflows 64 bits are refused, not wrapped
    to a small size, and a host pointer is refused before any launch (both
    entry points share the same argument checks)."""
    import paper_2210_07094_gb300 as df
    from paper_2210_07094_gb300 import _lib, synth

    L = _lib.load()
    m = df.Mechanism(synth.h2_air_mechanism())
    size = C.c_size_t(0)
    # 2^31 cells x (2^31 - 1) steps x 11 doubles x 8 bytes exceeds 2^64
    assert L.df_chem_adjoint_workspace_size(m.handle, 1 << 31, (1 << 31) - 1, C.byref(size)) == -5
    dev = torch.zeros(16, dtype=torch.float64, device=DEV)
    st = torch.zeros(16, dtype=torch.int32, device=DEV)
    rc = L.df_chem_adjoint_static(m.handle, 1 << 31, _ptr(dev), _ptr(dev), _ptr(dev), C.c_double(1e-6), None,
                                  (1 << 30), None, None, None, None, None, None, _ptr(st), None, None)
    assert rc == -5  # DF_EWORKSPACE, before anything is launched
    host = np.zeros(16)
    hp = C.c_void_p(host.ctypes.data)
    for fn in (L.df_chem_adjoint_static,):
        rc = fn(m.handle, 16, hp, _ptr(dev), _ptr(dev), C.c_double(1e-6), None, 4, None, None, None, None,
                None, None, _ptr(st), None, None)
        assert rc == -1  # DF_EINVAL: T0 is not device memory
    rc = L.df_chem_adjoint_static(m.handle, 16, _ptr(dev), _ptr(dev), _ptr(dev), C.c_double(1e-6), None, 4,
                                  hp, None, None, None, None, None, _ptr(st), None, None)
    assert rc == -1  # a cotangent in host memory
    buf = C.create_string_buffer(512)
    L.df_get_last_error_detail(buf, 512)
    assert b"gT1 must be device memory" in buf.value
