"""GB300-native per-cell chemistry substep (DeepFlame's CVODE / DNN hot path).

Python front end of ``libdfchem.so``: torch tensors in, device pointers to
the C ABI of ``include/df_chem.h``.  PyTorch provides device memory and
streams only; every step of the computation runs in the library's kernels.

    mech = Mechanism("mech.json")          # or a mechanism dict
    status, nsub = integrate(mech, T, p, Y, dt)   # T, Y updated in place
"""
from __future__ import annotations

import ctypes as C
import json
import os
import tempfile

from . import _lib

__all__ = ["Mechanism", "rhs", "jacobian", "integrate", "adjoint", "chem_step", "IntegOpts",
           "default_opts", "Dnn", "DnnOpts", "dnn_default_opts"]

IntegOpts = _lib.IntegOpts
default_opts = _lib.default_opts


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t, name, dtype=None, numel=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return C.c_void_p(t.data_ptr())


class Mechanism:
    """A loaded mechanism (species, reactions, thermo) resident on the device."""

    def __init__(self, src):
        lib = _lib.load()
        path = src
        tmp = None
        if isinstance(src, dict):
            fd, tmp = tempfile.mkstemp(suffix=".json")
            with os.fdopen(fd, "w") as f:
                json.dump(src, f)
            path = tmp
        h = C.c_void_p()
        try:
            _lib.check(lib.df_mech_load(os.fsencode(path), C.byref(h)), "df_mech_load")
        finally:
            if tmp:
                os.unlink(tmp)
        self._h = h
        ns, nr = C.c_int(), C.c_int()
        _lib.check(lib.df_mech_info(h, C.byref(ns), C.byref(nr)), "df_mech_info")
        self.n_species, self.n_reactions = ns.value, nr.value

    @property
    def handle(self):
        return self._h

    def set_lnA(self, lnA=None, stream=None):
        """Override ln A_j (device tensor of M doubles); None restores the file."""
        torch = _torch()
        ptr = None if lnA is None else _dptr(lnA, "lnA", torch.float64, self.n_reactions)
        _lib.check(_lib.load().df_mech_set_lnA(self._h, ptr, _stream_ptr(stream)), "df_mech_set_lnA")

    def last_stats(self, stream=None):
        a, r = C.c_int64(), C.c_int64()
        _lib.check(_lib.load().df_chem_last_stats(self._h, C.byref(a), C.byref(r), _stream_ptr(stream)),
                   "df_chem_last_stats")
        return a.value, r.value

    def jit_info(self):
        """(used, detail): whether the last thread-path integrator launch ran the
        kernel generated for this mechanism, and its state (compile time or
        why it is unavailable)."""
        used = C.c_int32()
        buf = C.create_string_buffer(4096)
        _lib.check(_lib.load().df_chem_jit_info(self._h, C.byref(used), buf, 4096), "df_chem_jit_info")
        return bool(used.value), buf.value.decode()

    def autotune(self, T, p, Y, dt: float, opts: IntegOpts | None = None, sample: int = 0, stream=None):
        """Time the integrator's launch shapes on (a copy of) the first `sample`
        cells and cache the fastest in the handle (df_chem_autotune).
        Returns (best IntegOpts, its time in ms)."""
        n, pT, pp, pY = _cells(self, T, p, Y)
        best = IntegOpts()
        ms = C.c_float()
        _lib.check(_lib.load().df_chem_autotune(self._h, n, pT, pp, pY, float(dt),
                                                C.byref(opts) if opts is not None else None, int(sample),
                                                C.byref(best), C.byref(ms), _stream_ptr(stream)),
                   "df_chem_autotune")
        return best, ms.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().df_mech_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _cells(mech, T, p, Y):
    torch = _torch()
    n = T.numel()
    return n, _dptr(T, "T", torch.float64), _dptr(p, "p", torch.float64, n), \
        _dptr(Y, "Y", torch.float64, mech.n_species * n)


def rhs(mech: Mechanism, T, p, Y, stream=None):
    """dy/dt [(N+1), ncells] and heat release [ncells] (W/m^3)."""
    torch = _torch()
    n, pT, pp, pY = _cells(mech, T, p, Y)
    dydt = torch.empty((mech.n_species + 1, n), dtype=torch.float64, device=T.device)
    qdot = torch.empty(n, dtype=torch.float64, device=T.device)
    _lib.check(_lib.load().df_chem_rhs(mech.handle, n, pT, pp, pY, _dptr(dydt, "dydt"), _dptr(qdot, "qdot"),
                                       _stream_ptr(stream)), "df_chem_rhs")
    return dydt, qdot


def jacobian(mech: Mechanism, T, p, Y, stream=None):
    """Analytic Jacobian [ncells, N+1, N+1] of (dT/dt, dY/dt) w.r.t. (T, Y)."""
    torch = _torch()
    n, pT, pp, pY = _cells(mech, T, p, Y)
    m = mech.n_species + 1
    J = torch.empty((n, m, m), dtype=torch.float64, device=T.device)
    _lib.check(_lib.load().df_chem_jacobian(mech.handle, n, pT, pp, pY, _dptr(J, "J"), _stream_ptr(stream)),
               "df_chem_jacobian")
    return J


def integrate(mech: Mechanism, T, p, Y, dt: float, opts: IntegOpts | None = None, status=None,
              nsub=None, stream=None):
    """Advance every cell over dt in place (T [ncells], Y [N, ncells]).
    Returns (status, nsub) int32 device tensors."""
    torch = _torch()
    n, pT, pp, pY = _cells(mech, T, p, Y)
    if status is None:
        status = torch.empty(n, dtype=torch.int32, device=T.device)
    if nsub is None:
        nsub = torch.empty(n, dtype=torch.int32, device=T.device)
    o = C.byref(opts) if opts is not None else None
    _lib.check(_lib.load().df_chem_integrate(mech.handle, n, pT, pp, pY, float(dt), o,
                                             _dptr(status, "status", torch.int32, n),
                                             _dptr(nsub, "nsub", torch.int32, n), _stream_ptr(stream)),
               "df_chem_integrate")
    return status, nsub


def integrate_steps(mech: Mechanism, T, p, Y, dt: float, nsteps: int, opts: IntegOpts | None = None,
                    status=None, nsub=None, t_ign=None, stream=None):
    """Advance every cell by nsteps consecutive steps of dt in place and return
    (status, nsub, t_ign): t_ign is the time of the largest dT/dt (the
    ignition delay of Sec. 4.1) per cell."""
    torch = _torch()
    n, pT, pp, pY = _cells(mech, T, p, Y)
    if status is None:
        status = torch.empty(n, dtype=torch.int32, device=T.device)
    if nsub is None:
        nsub = torch.empty(n, dtype=torch.int32, device=T.device)
    if t_ign is None:
        t_ign = torch.empty(n, dtype=torch.float64, device=T.device)
    o = C.byref(opts) if opts is not None else None
    _lib.check(_lib.load().df_chem_integrate_steps(mech.handle, n, pT, pp, pY, float(dt), int(nsteps), o,
                                                   _dptr(status, "status", torch.int32, n),
                                                   _dptr(nsub, "nsub", torch.int32, n),
                                                   _dptr(t_ign, "t_ign", torch.float64, n), _stream_ptr(stream)),
               "df_chem_integrate_steps")
    return status, nsub, t_ign


def adjoint(mech: Mechanism, T0, p, Y0, dt: float, gT1=None, gY1=None, gQ1=None,
            opts: IntegOpts | None = None, max_steps: int = 64, stream=None, store_stages: bool = True):
    """Discrete adjoint of integrate() (RODAS4, accepted steps frozen).

    Returns a dict with gT0 [ncells], gY0 [N, ncells], g_lnA [M] (summed over
    cells), status, nsub and the checkpoint workspace (uint8 device tensor whose
    leading doubles are [cell][step][T, Y..., h]).  store_stages=False passes
    the compact workspace (checkpoints and partials only): the reverse sweep
    then recomputes each step instead of reading its stored stages and LU
    factors, keeping n + 1 doubles per accepted step instead of 8n + n^2 + 1
    (n = N + 1).  Both give bitwise the same result."""
    torch = _torch()
    lib = _lib.load()
    n, pT, pp, pY = _cells(mech, T0, p, Y0)
    dev = T0.device
    size = C.c_size_t()
    _lib.check(lib.df_chem_adjoint_workspace_size(mech.handle, n, int(max_steps), C.byref(size)),
               "df_chem_adjoint_workspace_size")
    if not store_stages:
        N, M = mech.n_species, mech.n_reactions
        size = C.c_size_t(8 * (n * int(max_steps) * (N + 2) + (n + 15) // 16 * M) + 256)
    ws = torch.empty(size.value, dtype=torch.uint8, device=dev)
    out = {
        "gT0": torch.empty(n, dtype=torch.float64, device=dev),
        "gY0": torch.empty((mech.n_species, n), dtype=torch.float64, device=dev),
        "g_lnA": torch.empty(mech.n_reactions, dtype=torch.float64, device=dev),
        "status": torch.empty(n, dtype=torch.int32, device=dev),
        "nsub": torch.empty(n, dtype=torch.int32, device=dev),
        "workspace": ws,
    }

    def opt(t, name, numel):
        if t is None:
            return None
        t = t.contiguous()
        out["_keep_" + name] = t
        return _dptr(t, name, torch.float64, numel)

    o = C.byref(opts) if opts is not None else None
    _lib.check(lib.df_chem_adjoint(mech.handle, n, pT, pp, pY, float(dt), o, int(max_steps),
                                   opt(gT1, "gT1", n), opt(gY1, "gY1", mech.n_species * n),
                                   opt(gQ1, "gQ1", n), _dptr(out["gT0"], "gT0"), _dptr(out["gY0"], "gY0"),
                                   _dptr(out["g_lnA"], "g_lnA"), _dptr(out["status"], "status"),
                                   _dptr(out["nsub"], "nsub"), _dptr(ws, "workspace"), size.value,
                                   _stream_ptr(stream)), "df_chem_adjoint")
    for k in [k for k in out if k.startswith("_keep_")]:
        del out[k]
    return out


def _make_chem_step():
    torch = _torch()

    class ChemStep(torch.autograd.Function):
        """(T0, p, Y0, lnA) -> (T(dt), Y(dt), qdot(dt)); backward by the discrete adjoint."""

        @staticmethod
        def forward(ctx, T0, p, Y0, lnA, mech, dt, opts, max_steps):
            if opts is not None and opts.method != 0:
                raise ValueError("chem_step: the adjoint differentiates RODAS4 (opts.method = 0)")
            mech.set_lnA(lnA.detach().contiguous())
            T = T0.detach().clone()
            Y = Y0.detach().clone()
            status, _ = integrate(mech, T, p, Y, dt, opts)
            _, qdot = rhs(mech, T, p, Y)
            ctx.save_for_backward(T0.detach(), p, Y0.detach(), lnA.detach())
            ctx.mech, ctx.dt, ctx.opts, ctx.max_steps = mech, dt, opts, max_steps
            ctx.mark_non_differentiable(status)
            return T, Y, qdot, status

        @staticmethod
        def backward(ctx, gT, gY, gQ, _gs):
            T0, p, Y0, lnA = ctx.saved_tensors
            ctx.mech.set_lnA(lnA.contiguous())
            r = adjoint(ctx.mech, T0, p, Y0, ctx.dt, gT, gY, gQ, ctx.opts, ctx.max_steps)
            bad = int((r["status"] != 0).sum())
            if bad:
                raise RuntimeError(f"chem_step backward: {bad} cells failed in the adjoint (status != 0; "
                                   f"DF_CELL_MAXSTEPS means more than max_steps = {ctx.max_steps} accepted "
                                   "substeps: raise max_steps)")
            return r["gT0"], None, r["gY0"], r["g_lnA"], None, None, None, None

    return ChemStep


_chem_step = None


def chem_step(mech: Mechanism, T0, p, Y0, lnA, dt: float, opts: IntegOpts | None = None,
              max_steps: int = 64):
    """Differentiable chemistry substep: returns (T, Y, qdot, status).  Gradients
    flow to T0, Y0 and lnA (the natural logs of the pre-exponential factors).

    The forward pass runs df_chem_integrate with `opts` (RODAS4 only); the
    backward pass re-runs RODAS4 inside df_chem_adjoint and differentiates that
    run with its accepted steps held fixed.  The two evaluations of the rates
    agree to rounding, so both runs take the same steps except where a step
    sits exactly on the accept/reject boundary.  A cell that fails in the
    adjoint (e.g. more than max_steps accepted substeps) raises instead of
    returning a zero gradient."""
    global _chem_step
    if _chem_step is None:
        _chem_step = _make_chem_step()
    return _chem_step.apply(T0, p, Y0, lnA, mech, dt, opts, max_steps)


DnnOpts = _lib.DnnOpts


def dnn_default_opts() -> DnnOpts:
    o = DnnOpts()
    _lib.load().df_dnn_opts_default(C.byref(o))
    return o


class Dnn:
    """DNN chemistry integrator (Box-Cox features, 3 GELU hidden layers on the
    tensor cores, FP64 fallback to the integrator outside the training range)."""

    def __init__(self, opts: DnnOpts | None = None, seed: int = 22, _handle=None, n_species=None):
        lib = _lib.load()
        self._n_species = n_species if n_species is not None else (opts.n_species if opts is not None else 9)
        if _handle is not None:
            self._h = _handle
        else:
            h = C.c_void_p()
            _lib.check(lib.df_dnn_create(C.byref(opts) if opts is not None else None, int(seed), C.byref(h)),
                       "df_dnn_create")
            self._h = h
        self.n_params = lib.df_dnn_param_count(self._h)

    @classmethod
    def load(cls, path: str):
        import struct
        with open(path, "rb") as f:
            f.read(8)
            n_species = struct.unpack("<i", f.read(4))[0]
        h = C.c_void_p()
        _lib.check(_lib.load().df_dnn_load(os.fsencode(path), C.byref(h)), "df_dnn_load")
        return cls(_handle=h, n_species=n_species)

    def save(self, path: str):
        _lib.check(_lib.load().df_dnn_save(self._h, os.fsencode(path)), "df_dnn_save")

    def fit_norm(self, T, p, Y, Y_next, stream=None):
        torch = _torch()
        n = T.numel()
        _lib.check(_lib.load().df_dnn_fit_norm(self._h, n, _dptr(T, "T", torch.float64), _dptr(p, "p"),
                                               _dptr(Y, "Y"), _dptr(Y_next, "Y_next"), _stream_ptr(stream)),
                   "df_dnn_fit_norm")

    def norm(self):
        import numpy as np
        o = self.opts_n()
        arrs = [np.zeros(o + 2, np.float32), np.zeros(o + 2, np.float32), np.zeros(o, np.float32),
                np.zeros(o, np.float32), np.zeros(o + 2, np.float32), np.zeros(o + 2, np.float32)]
        ptrs = [a.ctypes.data_as(C.c_void_p) for a in arrs]
        _lib.check(_lib.load().df_dnn_get_norm(self._h, *ptrs), "df_dnn_get_norm")
        keys = ["mean_in", "std_in", "mean_out", "std_out", "in_min", "in_max"]
        return dict(zip(keys, arrs))

    def set_norm(self, **kw):
        import numpy as np
        keys = ["mean_in", "std_in", "mean_out", "std_out", "in_min", "in_max"]
        arrs = [None if kw.get(k) is None else np.ascontiguousarray(kw[k], np.float32) for k in keys]
        ptrs = [None if a is None else a.ctypes.data_as(C.c_void_p) for a in arrs]
        _lib.check(_lib.load().df_dnn_set_norm(self._h, *ptrs), "df_dnn_set_norm")

    def opts_n(self):
        # number of species, from the parameter layout
        return self._n_species

    def train_step(self, T, p, Y, Y_next, lr: float, want_loss: bool = True, stream=None):
        torch = _torch()
        n = T.numel()
        loss = C.c_float()
        _lib.check(_lib.load().df_dnn_train_step(self._h, n, _dptr(T, "T", torch.float64), _dptr(p, "p"),
                                                 _dptr(Y, "Y"), _dptr(Y_next, "Y_next"), float(lr),
                                                 C.byref(loss) if want_loss else None, _stream_ptr(stream)),
                   "df_dnn_train_step")
        return loss.value if want_loss else None

    def infer(self, mech: Mechanism, T, p, Y, dt: float, fallback_opts: IntegOpts | None = None,
              used_fallback=None, status=None, stream=None):
        """Advance cells in place with the network; returns (n_fallback, used_fallback, status)."""
        torch = _torch()
        n = T.numel()
        if used_fallback is None:
            used_fallback = torch.empty(n, dtype=torch.int32, device=T.device)
        if status is None:
            status = torch.empty(n, dtype=torch.int32, device=T.device)
        nfb = C.c_int64()
        _lib.check(_lib.load().df_dnn_infer(self._h, mech.handle, n, _dptr(T, "T", torch.float64),
                                            _dptr(p, "p", torch.float64, n),
                                            _dptr(Y, "Y", torch.float64, mech.n_species * n), float(dt),
                                            C.byref(fallback_opts) if fallback_opts is not None else None,
                                            _dptr(used_fallback, "used_fallback", torch.int32, n), C.byref(nfb),
                                            _dptr(status, "status", torch.int32, n), _stream_ptr(stream)),
                   "df_dnn_infer")
        return nfb.value, used_fallback, status

    def grad(self, T, p, Y, Y_next, n_total: int | None = None, want_loss: bool = True, stream=None):
        """Forward and backward pass without an update (df_dnn_grad): the
        gradient of this batch's share of a loss averaged over n_total rows
        (default: this batch) is left in grad_tensor().  Returns the loss share."""
        torch = _torch()
        n = T.numel()
        loss = C.c_float()
        _lib.check(_lib.load().df_dnn_grad(self._h, n, int(n_total if n_total is not None else n),
                                           _dptr(T, "T", torch.float64), _dptr(p, "p"), _dptr(Y, "Y"),
                                           _dptr(Y_next, "Y_next"), C.byref(loss) if want_loss else None,
                                           _stream_ptr(stream)), "df_dnn_grad")
        return loss.value if want_loss else None

    def grad_tensor(self):
        """The handle's FP32 gradient buffer as a CUDA tensor (no copy; valid
        while the handle lives), for an in-place all-reduce between grad()
        and adam_step()."""
        torch = _torch()
        ptr, cnt = C.c_void_p(), C.c_int64()
        _lib.check(_lib.load().df_dnn_grad_buffer(self._h, C.byref(ptr), C.byref(cnt)), "df_dnn_grad_buffer")

        class _Buf:
            __cuda_array_interface__ = {"shape": (cnt.value,), "typestr": "<f4", "data": (ptr.value, False),
                                        "version": 3, "strides": None}
        return torch.as_tensor(_Buf(), device=torch.device("cuda", torch.cuda.current_device()))

    def adam_step(self, lr: float, stream=None):
        """One Adam step with the gradient in grad_tensor() (df_dnn_adam_step)."""
        _lib.check(_lib.load().df_dnn_adam_step(self._h, float(lr), _stream_ptr(stream)), "df_dnn_adam_step")

    def adam_state(self):
        """(m1, m2, step): Adam's moment estimates (host float32) and step count."""
        import numpy as np
        m1 = np.zeros(self.n_params, np.float32)
        m2 = np.zeros(self.n_params, np.float32)
        st = C.c_int64()
        _lib.check(_lib.load().df_dnn_get_adam_state(self._h, m1.ctypes.data_as(C.c_void_p),
                                                     m2.ctypes.data_as(C.c_void_p), C.byref(st)),
                   "df_dnn_get_adam_state")
        return m1, m2, st.value

    def forward_raw(self, X, stream=None):
        """Network output U [n, 16] f32 for prepared bf16 features X [n, 16]."""
        torch = _torch()
        n = X.shape[0]
        U = torch.empty((n, 16), dtype=torch.float32, device=X.device)
        _lib.check(_lib.load().df_dnn_forward_raw(self._h, n, _dptr(X, "X", torch.bfloat16, n * 16),
                                                  _dptr(U, "U"), _stream_ptr(stream)), "df_dnn_forward_raw")
        return U

    def params(self):
        import numpy as np
        a = np.zeros(self.n_params, np.float32)
        _lib.check(_lib.load().df_dnn_get_params(self._h, a.ctypes.data_as(C.c_void_p)), "df_dnn_get_params")
        return a

    def grads(self):
        import numpy as np
        a = np.zeros(self.n_params, np.float32)
        _lib.check(_lib.load().df_dnn_get_grads(self._h, a.ctypes.data_as(C.c_void_p)), "df_dnn_get_grads")
        return a

    def set_params(self, a):
        import numpy as np
        a = np.ascontiguousarray(a, np.float32)
        assert a.size == self.n_params
        _lib.check(_lib.load().df_dnn_set_params(self._h, a.ctypes.data_as(C.c_void_p)), "df_dnn_set_params")

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().df_dnn_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
