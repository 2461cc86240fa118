"""The integrator kernel generated for a loaded mechanism (df_integ_opts.jit):
it runs on the thread-per-cell path at constant pressure, agrees with the
mechanism-independent kernel to rounding (the same operations in the same
order; the two compilations may contract different multiply-adds, which can
move a step-size decision that sits on the error threshold), follows
df_mech_set_lnA (the rate parameters stay in the blob), and agrees with the
oracle.  With jit = 1, and for the constant-volume reactor, the
mechanism-independent kernel runs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07094_gb300 as df  # noqa: E402
from oracle.oracle import Mech  # noqa: E402
from oracle.parity import check_integrator  # noqa: E402
from paper_2210_07094_gb300 import synth  # noqa: E402

DEV = "cuda:0"


def _dev(f):
    return (torch.tensor(f["T"], device=DEV), torch.tensor(f["p"], device=DEV),
            torch.tensor(np.ascontiguousarray(f["Y"]), device=DEV))


def _run(m, T0, p, Y0, dt, bt, jit, reactor=0):
    o = df.default_opts()
    o.block_threads, o.blocks_per_sm, o.path, o.jit, o.reactor = bt, 0, 1, jit, reactor
    T, Y = T0.clone(), Y0.clone()
    st, ns = df.integrate(m, T, p, Y, dt, o)
    used, detail = m.jit_info()
    return (T, Y, st, ns), used, detail


def _close(a, b):
    """Same statuses; T within 1e-6 K and Y within 1e-9 of the cell's largest
    mass fraction (the integrator's own error against the oracle is ~1e-7 K);
    at most 1% of the cells with another number of substeps."""
    (T1, Y1, s1, n1), (T2, Y2, s2, n2) = a, b
    assert torch.equal(s1, s2)
    dT = (T1 - T2).abs().max().item()
    dY = ((Y1 - Y2).abs() / Y1.abs().amax(dim=0)).max().item()
    moved = (n1 != n2).float().mean().item()
    assert dT <= 1e-6 and dY <= 1e-9 and moved <= 0.01, (dT, dY, moved)
    return dT, dY, moved


@pytest.fixture(scope="module")
def h2():
    mech = synth.h2_air_mechanism()
    return mech, df.Mechanism(mech)


def test_generated_kernel_runs_and_matches_the_generic_kernel(h2):
    mech, m = h2
    f = synth.field(1, mech, 12000, seed=77)
    T0, p, Y0 = _dev(f)
    ref, used, _ = _run(m, T0, p, Y0, f["dt"], 32, 1)
    assert not used and int(ref[2].abs().sum()) == 0
    for bt in (32, 64):
        out, used, detail = _run(m, T0, p, Y0, f["dt"], bt, 0)
        assert used, detail
        assert "compiled" in detail or "cache" in detail
        print("generated vs mechanism-independent", bt, _close(ref, out))
    # block sizes without a generated kernel run the mechanism-independent one
    out, used, _ = _run(m, T0, p, Y0, f["dt"], 128, 0)
    assert not used and all(torch.equal(x, y) for x, y in zip(ref, out))


def test_generated_kernel_follows_set_lnA(h2):
    mech, m = h2
    f = synth.field(0, mech, 3000, seed=78)
    T0, p, Y0 = _dev(f)
    rng = np.random.default_rng(3)
    lnA0 = np.log([r["A"] for r in mech["reactions"]])
    lnA = torch.tensor(lnA0 + rng.uniform(-0.5, 0.5, lnA0.size), device=DEV)
    m.set_lnA(lnA)
    try:
        ref, _, _ = _run(m, T0, p, Y0, f["dt"], 64, 1)
        out, used, detail = _run(m, T0, p, Y0, f["dt"], 64, 0)
        assert used, detail
        _close(ref, out)
    finally:
        m.set_lnA(None)
    base, used, _ = _run(m, T0, p, Y0, f["dt"], 64, 0)
    assert used and not torch.equal(base[0], out[0])


def test_generated_kernel_matches_the_oracle(h2):
    mech, m = h2
    o = Mech(mech)
    f = synth.field(0, mech, 600, seed=79)
    T0, p, Y0 = _dev(f)
    (T, Y, st, _), used, detail = _run(m, T0, p, Y0, f["dt"], 32, 0)
    assert used, detail
    assert int(st.abs().sum()) == 0
    To, Yo, so, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"])
    assert np.all(so == 0)
    print(check_integrator(f["T"], f["Y"], T.cpu().numpy(), Y.cpu().numpy(), To, Yo))


def test_three_species_mechanism_and_constant_volume():
    mech = synth.isomer_mechanism()
    m = df.Mechanism(mech)
    n = 700
    T0 = torch.full((n,), 1100.0, dtype=torch.float64, device=DEV)
    p = torch.full((n,), 101325.0, dtype=torch.float64, device=DEV)
    Y0 = torch.zeros((m.n_species, n), dtype=torch.float64, device=DEV)
    Y0[0] = torch.linspace(0.1, 0.9, n, dtype=torch.float64, device=DEV)
    Y0[1] = 0.05
    Y0[2] = 1.0 - Y0[0] - Y0[1]
    ref, used, _ = _run(m, T0, p, Y0, 1e-5, 64, 1)
    out, used, detail = _run(m, T0, p, Y0, 1e-5, 64, 0)
    assert used, detail
    _close(ref, out)
    # the constant-volume reactor has no generated kernel
    _, used, _ = _run(m, T0, p, Y0, 1e-5, 64, 0, reactor=1)
    assert not used


def test_thread_path_for_a_species_count_without_a_built_kernel():
    """14 species (no compiled thread kernel): with jit the automatic path runs
    the generated thread-per-cell kernel; it agrees with the warp path and the
    oracle; with jit = 1 the automatic path is the warp path and an explicit
    thread path is refused."""
    mech = synth.hydrocarbon_mechanism(n_species=12, M=40, n_tb=4, n_troe=2)
    m = df.Mechanism(mech)
    assert m.n_species == 14
    f = synth.field(2, mech, 300, seed=5)
    T0, p, Y0 = _dev(f)
    T, Y = T0.clone(), Y0.clone()
    st, _ = df.integrate(m, T, p, Y, f["dt"])
    used, detail = m.jit_info()
    assert used, detail
    assert int(st.abs().sum()) == 0
    o = df.default_opts()
    o.path = 2
    Tw, Yw = T0.clone(), Y0.clone()
    df.integrate(m, Tw, p, Yw, f["dt"], o)
    assert torch.max(torch.abs(T - Tw)).item() <= 1e-6
    assert torch.max(torch.abs(Y - Yw)).item() <= 1e-10
    idx = np.arange(0, 300, 5)
    To, Yo, so, _ = Mech(mech).integrate(f["T"][idx], f["p"][idx], f["Y"][:, idx], f["dt"])
    assert np.all(so == 0)
    print(check_integrator(f["T"][idx], f["Y"][:, idx], T.cpu().numpy()[idx], Y.cpu().numpy()[:, idx], To, Yo))
    o = df.default_opts()
    o.jit = 1
    Tg, Yg = T0.clone(), Y0.clone()
    df.integrate(m, Tg, p, Yg, f["dt"], o)
    assert not m.jit_info()[0]
    assert torch.equal(Tg, Tw) and torch.equal(Yg, Yw)
    o.path = 1
    with pytest.raises(df._lib.DFError):
        df.integrate(m, T0.clone(), p, Y0.clone(), f["dt"], o)
    # the autotuner weighs the generated thread kernel against the warp path
    best, ms = m.autotune(T0, p, Y0, f["dt"])
    assert best.path in (1, 2) and ms > 0


_CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_2210_07094_gb300 as df
from paper_2210_07094_gb300 import synth
mech = synth.isomer_mechanism(kind="three-body", A=3e10, eff={"D": 2.5})
m = df.Mechanism(mech)
n = 64
T = torch.full((n,), 1250.0, dtype=torch.float64, device="cuda")
p = torch.full((n,), 101325.0, dtype=torch.float64, device="cuda")
Y = torch.tensor(np.tile([[0.6], [0.1], [0.3]], (1, n)), device="cuda")
df.integrate(m, T, p, Y, 1e-6)
used, detail = m.jit_info()
print(json.dumps({"used": used, "detail": detail, "Y0": Y[0].cpu().tolist()}))
"""


def test_compiled_module_is_cached_on_disk(tmp_path):
    """A second process finds the module the first one compiled in the cache
    directory (DF_JIT_CACHE) and gives bitwise the same cells."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, DF_JIT_CACHE=str(tmp_path / "cache"))
    out = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", _CHILD, root], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        out.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert out[0]["used"] and "compiled" in out[0]["detail"], out[0]["detail"]
    assert out[1]["used"] and "cache" in out[1]["detail"], out[1]["detail"]
    assert out[0]["Y0"] == out[1]["Y0"]
    assert sorted(os.listdir(tmp_path / "cache"))[0].endswith(".cubin")

