"""ctypes binding of ``libdfchem.so`` (the C ABI declared in ``include/df_chem.h``).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  There is no fallback: if the library is missing or cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdfchem.so")

DF_OK = 0
ERRORS = {-1: "DF_EINVAL", -2: "DF_ENOMEM", -3: "DF_ECUDA", -4: "DF_EMECH", -5: "DF_EWORKSPACE",
          -6: "DF_ETIMEOUT", -7: "DF_EUNSUPPORTED"}
CELL_OK, CELL_MAXSTEPS, CELL_NONFINITE, CELL_HMIN = 0, 1, 2, 3


class IntegOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol_Y", C.c_double), ("atol_T", C.c_double),
                ("h0", C.c_double), ("h_min", C.c_double), ("max_substeps", C.c_int32),
                ("method", C.c_int32), ("block_threads", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("order_by_T", C.c_int32), ("path", C.c_int32), ("reactor", C.c_int32),
                ("jit", C.c_int32)]


class DnnOpts(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("width", C.c_int32 * 3), ("lambda_", C.c_double),
                ("batch", C.c_int32), ("infer_chunk", C.c_int32), ("beta1", C.c_double),
                ("beta2", C.c_double), ("adam_eps", C.c_double), ("range_margin", C.c_double),
                ("reserved", C.c_int32 * 4)]


class DFError(RuntimeError):
    def __init__(self, code: int, fn: str, detail: str):
        super().__init__(f"{fn} failed: {ERRORS.get(code, code)}: {detail}")
        self.code = code


_lib = None

# (name, restype, argtypes) of every exported symbol
_p, _i, _d, _i64, _sz = C.c_void_p, C.c_int, C.c_double, C.c_int64, C.c_size_t
SIGNATURES = [
    ("df_integ_opts_default", None, [_p]),
    ("df_mech_load", _i, [C.c_char_p, _p]),
    ("df_mech_free", None, [_p]),
    ("df_mech_info", _i, [_p, _p, _p]),
    ("df_mech_set_lnA", _i, [_p, _p, _p]),
    ("df_chem_rhs", _i, [_p, _i64, _p, _p, _p, _p, _p, _p]),
    ("df_chem_jacobian", _i, [_p, _i64, _p, _p, _p, _p, _p]),
    ("df_chem_integrate", _i, [_p, _i64, _p, _p, _p, _d, _p, _p, _p, _p]),
    ("df_chem_last_stats", _i, [_p, _p, _p, _p]),
    ("df_chem_jit_info", _i, [_p, _p, C.c_char_p, _sz]),
    ("df_mech_generated_source", _i, [C.c_char_p, C.c_char_p, _sz, _p]),
    ("df_chem_autotune", _i, [_p, _i64, _p, _p, _p, _d, _p, _i64, _p, _p, _p]),
    ("df_chem_integrate_steps", _i, [_p, _i64, _p, _p, _p, _d, C.c_int32, _p, _p, _p, _p, _p]),
    ("df_chem_adjoint_workspace_size", _i, [_p, _i64, C.c_int32, _p]),
    ("df_chem_adjoint", _i, [_p, _i64, _p, _p, _p, _d, _p, C.c_int32, _p, _p, _p, _p, _p, _p, _p, _p,
                             _p, _sz, _p]),
    ("df_chem_adjoint_static", _i, [_p, _i64, _p, _p, _p, _d, _p, C.c_int32, _p, _p, _p, _p, _p, _p, _p, _p,
                                    _p]),
    ("df_dnn_opts_default", None, [_p]),
    ("df_dnn_create", _i, [_p, C.c_uint64, _p]),
    ("df_dnn_free", None, [_p]),
    ("df_dnn_set_norm", _i, [_p, _p, _p, _p, _p, _p, _p]),
    ("df_dnn_get_norm", _i, [_p, _p, _p, _p, _p, _p, _p]),
    ("df_dnn_fit_norm", _i, [_p, _i64, _p, _p, _p, _p, _p]),
    ("df_dnn_train_step", _i, [_p, _i64, _p, _p, _p, _p, C.c_float, _p, _p]),
    ("df_dnn_grad", _i, [_p, _i64, _i64, _p, _p, _p, _p, _p, _p]),
    ("df_dnn_grad_buffer", _i, [_p, _p, _p]),
    ("df_dnn_adam_step", _i, [_p, C.c_float, _p]),
    ("df_dnn_get_adam_state", _i, [_p, _p, _p, _p]),
    ("df_dnn_infer", _i, [_p, _p, _i64, _p, _p, _p, _d, _p, _p, _p, _p, _p]),
    ("df_dnn_forward_raw", _i, [_p, _i64, _p, _p, _p]),
    ("df_dnn_param_count", _i64, [_p]),
    ("df_dnn_get_params", _i, [_p, _p]),
    ("df_dnn_set_params", _i, [_p, _p]),
    ("df_dnn_get_grads", _i, [_p, _p]),
    ("df_dnn_save", _i, [_p, C.c_char_p]),
    ("df_dnn_load", _i, [C.c_char_p, _p]),
    ("df_strerror", C.c_char_p, [_i]),
    ("df_get_last_error_detail", _i, [C.c_char_p, _sz]),
    ("df_probe_fp64_peak", _i, [_i, _p, _p]),
    ("df_probe_fp64_chains", _i, [_i, _i, _i, _p, _p]),
    ("df_probe_exp", _i, [_p, _p, C.c_longlong, _i, _p]),
    ("df_probe_gelu", _i, [_p, _p, C.c_longlong, _i, _p]),
    ("df_probe_log", _i, [_p, _p, C.c_longlong, _p]),
    ("df_probe_gemm_bf16", _i, [_p, _p, _p, _i, _i, _i, _i, _p, _p]),
]


def load(path: str | None = None):
    """Load the library (once).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int, fn: str):
    if rc != DF_OK:
        buf = C.create_string_buffer(1024)
        load().df_get_last_error_detail(buf, 1024)
        raise DFError(rc, fn, buf.value.decode(errors="replace"))


def default_opts() -> IntegOpts:
    o = IntegOpts()
    load().df_integ_opts_default(C.byref(o))
    return o
