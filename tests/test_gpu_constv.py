"""Constant-volume reactor (Sec. 2.2, df0DFoam's constant-volume case): the
GPU integrator with reactor = 1 against the oracle's constant-volume
integration, on both kernel paths."""
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


def _cv():
    o = df.default_opts()
    o.reactor = 1
    return o


@pytest.fixture(scope="module")
def h2():
    mech = synth.h2_air_mechanism()
    return mech, df.Mechanism(mech), Mech(mech)


@pytest.mark.parametrize("cfg,n", [(0, 1000), (1, 600)])
def test_constant_volume_matches_oracle(h2, cfg, n):
    mech, m, o = h2
    f = synth.field(cfg, mech, n, seed=70 + cfg)
    T, p, Y = _dev(f)
    st, _ = df.integrate(m, T, p, Y, f["dt"], _cv())
    To, Yo, so, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"], constant_volume=True)
    assert int(st.abs().sum()) == 0 and np.all(so == 0)
    Tg, Yg = T.cpu().numpy(), Y.cpu().numpy()
    print(check_integrator(f["T"], f["Y"], Tg, Yg, To, Yo))
    # internal energy conserved, and the heat goes into cv: more heating than at
    # constant pressure wherever the constant-pressure run heats noticeably
    for c in range(0, n, 97):
        u0 = o.internal_energy_mass(f["T"][c], f["Y"][:, c])
        u1 = o.internal_energy_mass(Tg[c], Yg[:, c])
        assert abs(u1 - u0) <= 1e-7 * 1.5e3 * f["T"][c]
    T2, p2, Y2 = _dev(f)
    df.integrate(m, T2, p2, Y2, f["dt"])
    dTp = T2.cpu().numpy() - f["T"]
    dTv = Tg - f["T"]
    big = dTp > 0.05
    if big.any():
        assert np.all(dTv[big] > dTp[big])


def test_constant_volume_warp_path():
    mech = synth.hydrocarbon_mechanism()
    m, o = df.Mechanism(mech), Mech(mech)
    f = synth.field(2, mech, 24, seed=77)
    T, p, Y = _dev(f)
    st, _ = df.integrate(m, T, p, Y, f["dt"], _cv())
    To, Yo, so, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"], constant_volume=True)
    assert int(st.abs().sum()) == 0 and np.all(so == 0)
    print(check_integrator(f["T"], f["Y"], T.cpu().numpy(), Y.cpu().numpy(), To, Yo))
    # the 9-species mechanism on the warp path agrees with the thread path
    mech9 = synth.h2_air_mechanism()
    m9 = df.Mechanism(mech9)
    g = synth.field(1, mech9, 200, seed=78)
    Ta, pa, Ya = _dev(g)
    Tb, pb, Yb = _dev(g)
    ow = _cv()
    ow.path = 2
    df.integrate(m9, Ta, pa, Ya, g["dt"], _cv())
    df.integrate(m9, Tb, pb, Yb, g["dt"], ow)
    assert torch.max(torch.abs(Ta - Tb)).item() <= 1e-6
    assert torch.max(torch.abs(Ya - Yb)).item() <= 1e-10


def test_constant_volume_multistep_and_unsupported_calls(h2):
    mech, m, o = h2
    f = synth.field(1, mech, 500, seed=79)
    T, p, Y = _dev(f)
    T2, Y2 = T.clone(), Y.clone()
    st, ns, ti = df.integrate_steps(m, T, p, Y, f["dt"], 1, _cv())
    df.integrate(m, T2, p, Y2, f["dt"], _cv())
    assert torch.equal(T, T2) and torch.equal(Y, Y2)
    from paper_2210_07094_gb300 import _lib
    with pytest.raises(_lib.DFError):
        df.adjoint(m, T, p, Y, f["dt"], gT1=torch.ones_like(T), opts=_cv())
