"""The mechanism-specific integrator source (df_mech_generated_source) on the
host: one straight-line block per reaction with the mechanism's species
indices, the mechanism's numbers as its literals, and a source that NVRTC
compiles for sm_103a with the library's device headers (skipped when the
NVRTC library is absent)."""
import ctypes as C
import os
import re

import numpy as np
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
    # every species a reaction changes (net stoichiometric coefficient nonzero)
    # appears as a literal production-rate index; one it leaves unchanged
    # (O in O2 + H + O <=> O + HO2) does not
    for j, r in enumerate(mech["reactions"]):
        body = src.split(f"// reaction {j}\n")[1].split("// reaction")[0].split("double Hw")[0]
        for k in set(r["reactants"]) | set(r["products"]):
            net = r["products"].get(k, 0) - r["reactants"].get(k, 0)
            assert (f"wdot[{names.index(k)}]" in body) == (net != 0), (j, k, net)


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
    # the options the library compiles the module with (the 256-entry exp table)
    opts = [b"--gpu-architecture=sm_103a", b"-std=c++17", b"-I" + CSRC.encode(), b"-default-device",
            b"-diag-suppress=177", b"-DDF_EXP_TABLE_BITS=8"]
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


_HEX = re.compile(r"\((-?0x[0-9a-fA-F.]+p[+-]?\d+)\)")


def _lits(line):
    return [float.fromhex(x) for x in _HEX.findall(line)]


def test_generated_literals_are_the_mechanism_numbers(tmp_path):
    """The numbers the generator writes as literals are the mechanism's:
    NASA-7 coefficients (cp/R, h/RT and s/R polynomials, exactly-zero terms
    dropped), 1/W, W, beta, Ea/R, third-body efficiencies and Troe records."""
    mech = synth.h2_air_mechanism()
    src = _source(mech, tmp_path)
    R = 8.314462618
    for k, sp in enumerate(mech["species"]):
        a = sp["nasa7"]
        blk = src.split(f"// species {k}\n")[1].split("}")[0]
        # cp_k / (R W_k): the cp/R coefficients times the double 1 / W_k
        cp = _lits([ln for ln in blk.splitlines() if "cpw =" in ln][0])
        top = max(i for i in range(5) if a[i] != 0.0 or i == 0)
        assert cp == [c * (1.0 / sp["W"]) for c in a[: top + 1]]
        h = _lits([ln for ln in blk.splitlines() if "hk =" in ln][0])
        hpoly = [a[0]] + [a[i] / (i + 1) for i in range(1, 5)]
        htop = max(i for i in range(5) if hpoly[i] != 0.0 or i == 0)
        assert h == pytest.approx(hpoly[: htop + 1] + [a[5]], rel=1e-15)
        # g/RT = h/RT - s/R as one polynomial: (a1 - a7) - a1 ln T
        # + T (-a2/2 - a3 T/6 - a4 T^2/12 - a5 T^3/20) + a6 / T
        g = _lits([ln for ln in blk.splitlines() if "gk =" in ln][0])
        gpoly = [-a[1] / 2.0, -a[2] / 6.0, -a[3] / 12.0, -a[4] / 20.0]
        gtop = max(i for i in range(4) if gpoly[i] != 0.0 or i == 0)
        assert g == pytest.approx([a[0] - a[6], -a[0]] + gpoly[: gtop + 1] + [a[5]], rel=1e-15)
        iw = _lits([ln for ln in blk.splitlines() if "sumYW +=" in ln][0])
        assert iw == [pytest.approx(1.0 / sp["W"], rel=1e-15)]
        fl = [ln for ln in src.splitlines() if ln.strip().startswith(f"f[{1 + k}] =")][0]
        assert _lits(fl) == [sp["W"]]
    names = [s["name"] for s in mech["species"]]
    for j, r in enumerate(mech["reactions"]):
        blk = src.split(f"// reaction {j}\n")[1].split("// reaction")[0]
        beta = _lits([ln for ln in blk.splitlines() if "g.beta =" in ln][0])
        ear = _lits([ln for ln in blk.splitlines() if "g.EaR =" in ln][0])
        assert beta == [r["b"]]
        assert ear == [pytest.approx(r["Ea"] * 1e3 / R, rel=1e-15)]
        if r["type"] != "elementary":
            # [M] = sum of all C plus (eps_l - 1) C_l for every eps_l != 1
            assert "double Mc = ctot;" in blk
            mc = [_lits(ln)[0] for ln in blk.splitlines() if "Mc +=" in ln]
            eff = [r.get("efficiencies", {}).get(nm, 1.0) for nm in names]
            assert mc == [e - 1.0 for e in eff if e != 1.0]
        if r["type"] == "falloff-troe":
            trp = _lits([ln for ln in blk.splitlines() if "trp[" in ln][0])
            lo, tr = r["low"], r["troe"]
            expect = [np.log(lo["A"]) - np.log(r["A"]), lo["b"], lo["Ea"] * 1e3 / R, tr["alpha"],
                      1.0 / tr["T3"], 1.0 / tr["T1"], tr["T2"], 0.0]
            assert trp == pytest.approx(expect, rel=1e-14, abs=1e-300)


def test_generated_jacobian_entries_are_prescaled(tmp_path):
    """The Jacobian entries the generator writes: row k (a species the reaction
    changes, net coefficient nu_k) gets d q / d C_l scaled by nu_k W_k / W_l,
    the column scaling of the conversion to mass fractions; a third-body or
    falloff reaction adds nu_k d q / d[M] to the row's unit sum sM[k] and enters
    only the efficiencies that are not 1, as (eps_l - 1) W_k / W_l."""
    mech = synth.h2_air_mechanism()
    src = _source(mech, tmp_path)
    names = [s["name"] for s in mech["species"]]
    N = len(names)
    n = N + 1
    W = [s["W"] for s in mech["species"]]
    iW = [1.0 / w for w in W]
    for j, r in enumerate(mech["reactions"]):
        blk = src.split(f"// reaction {j}\n")[1].split("// reaction")[0].split("double Hw")[0]
        jac = blk.split("if (WITH_J) {")[1]
        nu = {}
        for sp_, v in r["reactants"].items():
            nu[names.index(sp_)] = nu.get(names.index(sp_), 0) - v
        for sp_, v in r["products"].items():
            nu[names.index(sp_)] = nu.get(names.index(sp_), 0) + v
        species = sorted(set(names.index(x) for x in list(r["reactants"]) + list(r["products"])))
        for k, vk in nu.items():
            if vk == 0:
                continue
            row = (1 + k) * n
            for l in species:
                if l == k:
                    continue
                lines = [ln for ln in jac.splitlines() if f"Jv[{row + 1 + l}] +=" in ln and f"* dq{l};" in ln]
                assert len(lines) == 1, (j, k, l)
                assert _lits(lines[0]) == [vk * (W[k] * iW[l])]
            if r["type"] != "elementary":
                assert f"sM[{k}] += cM;" in jac
                eff = [r.get("efficiencies", {}).get(nm, 1.0) for nm in names]
                cm = jac.split(f"sM[{k}] += cM;")[1].split("}")[0]
                got = {int(m.group(1)) - row - 1: _lits(m.group(0))[0]
                       for m in re.finditer(r"Jv\[(\d+)\] \+= cM \* (\(-?0x[0-9a-fA-F.]+p[+-]?\d+\))", cm)}
                want = {l: (eff[l] - 1.0) * (1.0 if l == k else W[k] * iW[l]) for l in range(N) if eff[l] != 1.0}
                assert got == want, (j, k)
