"""The mechanism-specific integrator source (df_mech_generated_source) on the
host: one straight-line block per reaction with the mechanism's species
indices, and a source that NVRTC compiles for sm_103a with the library's
device headers (skipped when the NVRTC library is absent)."""
import ctypes as C
import os
import re

import pytest

from paper_2210_07094_gb300 import _lib, synth

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2210_07094_gb300", "csrc")


def _source(mech, tmp_path):
    path = str(tmp_path / "mech.json")
    synth.write_json(mech, path)
    L = _lib.load()
    need = C.c_size_t()
    _lib.check(L.df_mech_generated_source(path.encode(), None, 0, C.byref(need)), "df_mech_generated_source")
    buf = C.create_string_buffer(need.value)
    _lib.check(L.df_mech_generated_source(path.encode(), buf, need.value, None), "df_mech_generated_source")
    return buf.value.decode()


def test_generated_source_has_one_block_per_reaction(tmp_path):
    mech = synth.h2_air_mechanism()
    src = _source(mech, tmp_path)
    assert "gen_eval" in src and "struct GenEval" in src
    blocks = re.findall(r"// reaction (\d+)\n", src)
    assert [int(b) for b in blocks] == list(range(len(mech["reactions"])))
    names = [s["name"] for s in mech["species"]]
    # every species a reaction changes appears as a literal production-rate index
    for j, r in enumerate(mech["reactions"]):
        body = src.split(f"// reaction {j}\n")[1].split("// reaction")[0]
        for k in list(r["reactants"]) + list(r["products"]):
            assert f"wdot[{names.index(k)}]" in body, (j, k)


def test_generated_source_rejects_a_bad_file(tmp_path):
    L = _lib.load()
    bad = tmp_path / "bad.json"
    bad.write_text("{}")
    assert L.df_mech_generated_source(str(bad).encode(), None, 0, None) == -4  # DF_EMECH


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so"):
        try:
            return C.CDLL(name)
        except OSError:
            continue
    return None


def test_generated_source_compiles_with_nvrtc(tmp_path):
    nv = _nvrtc()
    if nv is None:
        pytest.skip("NVRTC library not available")
    src = _source(synth.h2_air_mechanism(), tmp_path).encode()
    prog = C.c_void_p()
    assert nv.nvrtcCreateProgram(C.byref(prog), src, b"df_generated.cu", 0, None, None) == 0
    names = [b"df::k_integrate_thread<9, false, 32, df::GenEval>", b"&df::c_tab"]
    for nm in names:
        assert nv.nvrtcAddNameExpression(prog, nm) == 0
    opts = [b"--gpu-architecture=sm_103a", b"-std=c++17", b"-I" + CSRC.encode(), b"-default-device",
            b"-diag-suppress=177"]
    rc = nv.nvrtcCompileProgram(prog, len(opts), (C.c_char_p * len(opts))(*opts))
    n = C.c_size_t()
    nv.nvrtcGetProgramLogSize(prog, C.byref(n))
    log = C.create_string_buffer(n.value)
    nv.nvrtcGetProgramLog(prog, log)
    assert rc == 0, log.value.decode()[:3000]
    for nm in names:
        low = C.c_char_p()
        assert nv.nvrtcGetLoweredName(prog, nm, C.byref(low)) == 0 and low.value
    nv.nvrtcDestroyProgram(C.byref(prog))
