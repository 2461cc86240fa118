"""Multi-step driver (df_chem_integrate_steps): nsteps consecutive steps of dt
in one launch, and the ignition delay from [dT/dt]_max (Sec. 4.1), against
df_chem_integrate and the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07094_gb300 as df  # noqa: E402
from oracle.oracle import Mech  # noqa: E402
from paper_2210_07094_gb300 import synth  # noqa: E402

DEV = "cuda:0"


def _dev(T, p, Y):
    return (torch.tensor(T, device=DEV), torch.tensor(p, device=DEV),
            torch.tensor(np.ascontiguousarray(Y), device=DEV))


@pytest.fixture(scope="module")
def h2():
    mech = synth.h2_air_mechanism()
    return mech, df.Mechanism(mech), Mech(mech)


def test_one_step_equals_integrate(h2):
    mech, m, _ = h2
    f = synth.field(1, mech, 3000, seed=8)
    T, p, Y = _dev(f["T"], f["p"], f["Y"])
    T2, Y2 = T.clone(), Y.clone()
    st, ns = df.integrate(m, T, p, Y, f["dt"])
    st2, ns2, ti = df.integrate_steps(m, T2, p, Y2, f["dt"], 1)
    assert torch.equal(T, T2) and torch.equal(Y, Y2)
    assert torch.equal(st, st2) and torch.equal(ns, ns2)
    assert bool(((ti >= 0) & (ti < f["dt"])).all())


def test_ignition_window_against_oracle(h2):
    """Stoichiometric mixtures at 10 atm, T0 = 950..1200 K, 150 steps of 2 ms
    (the synthetic mechanism's heat release peaks 20-90 ms in): the final
    state matches the oracle, and the time of the largest dT/dt agrees within
    the sampling resolution (the rate peak is broad)."""
    mech, m, o = h2
    n = 24
    T0 = np.linspace(950.0, 1200.0, n)
    Y0 = np.asarray(synth._h2_air_Y(mech, np.ones(n)))
    p0 = np.full(n, 10 * 101325.0)
    dt, nsteps = 2e-3, 150
    T, p, Y = _dev(T0, p0, Y0)
    st, ns, ti = df.integrate_steps(m, T, p, Y, dt, nsteps)
    assert int(st.abs().sum()) == 0
    To, Yo, to, rate = o.ignition(T0, p0, Y0, dt, nsteps, grid=16)
    Tg, Yg = T.cpu().numpy(), Y.cpu().numpy()
    assert np.max(np.abs(Tg - To)) <= 1e-3
    assert np.max(np.abs(Yg - Yo) / Yo.max(axis=0)) <= 1e-7
    tig = ti.cpu().numpy()
    assert np.all(to > 5 * dt)  # an interior maximum, not the initial state
    # the oracle's grid resolves dt/16; the GPU's time is the vertex of the
    # parabola through its largest substep-start sample and the neighbours
    print({"max_abs_dt_ign_over_dt": float(np.max(np.abs(tig - to)) / dt)})
    assert np.all(np.abs(tig - to) <= dt / 4), np.max(np.abs(tig - to))
    # the GPU's chosen time has (nearly) the oracle's largest rate
    for c in range(0, n, 6):
        Tc, Yc, _, _ = o.integrate(T0[c:c + 1], p0[c:c + 1], Y0[:, c:c + 1], float(tig[c])) \
            if tig[c] > 0 else (T0[c:c + 1], Y0[:, c:c + 1], None, None)
        fT = o.rhs(p0[c], np.r_[Tc[0], Yc[:, 0]])[0][0]
        assert fT >= 0.999 * rate[c], (c, fT, rate[c])


def test_steps_match_repeated_calls_warp_path():
    mech = synth.hydrocarbon_mechanism()
    m = df.Mechanism(mech)
    f = synth.field(2, mech, 40, seed=12)
    T, p, Y = _dev(f["T"], f["p"], f["Y"])
    T2, Y2 = T.clone(), Y.clone()
    st, ns, ti = df.integrate_steps(m, T, p, Y, f["dt"], 3)
    for _ in range(3):
        df.integrate(m, T2, p, Y2, f["dt"])
    assert int(st.abs().sum()) == 0
    assert torch.max(torch.abs(T - T2)).item() <= 1e-4
    assert torch.max(torch.abs(Y - Y2)).item() <= 1e-8
    assert bool(((ti >= 0) & (ti < 3 * f["dt"])).all())


def test_ignition_time_of_the_logistic_closed_form():
    """A + B -> 2 B (equal W and cp, small heat of reaction): the largest dT/dt
    falls where Y_A = Y_B, at t* = ln(Y_A0 / Y_B0) / (r (Y_A0 + Y_B0)), r = A rho / W
    (the oracle reaches it within half its grid, CPU test).  The GPU's refined
    time lies within dt/20 of t*, far inside its substep spacing; the thread
    path (the 3-species built kernel) and the warp path agree."""
    mech = synth.autocatalytic_mechanism()
    m = df.Mechanism(mech)
    YA = np.array([0.5, 0.5, 0.3, 0.6] * 8)
    YB = np.array([1e-3, 1e-4, 1e-3, 5e-3] * 8)
    Y0 = np.vstack([YA, YB, 1.0 - YA - YB])
    n = YA.size
    rho = 10 * 101325.0 * 30.0 / (8.314462618e7 * 1000.0)
    tstar = np.log(YA / YB) / (1e7 * rho / 30.0 * (YA + YB))
    dt = 0.01
    for path in (1, 2):
        T, p, Y = _dev(np.full(n, 1000.0), np.full(n, 101325.0), Y0)
        o = df.default_opts()
        o.path = path
        st, ns, ti = df.integrate_steps(m, T, p, Y, dt, 25, o)
        assert int(st.abs().sum()) == 0
        err = np.abs(ti.cpu().numpy() - tstar)
        print({"path": path, "max_err_over_dt": float(err.max() / dt),
               "substeps_per_step": float(ns.float().mean() / 25)})
        assert np.all(err <= dt / 20), (path, err.max() / dt)
