"""Closed-form reaction cases on the GPU, through both thread-path kernels
(the one generated for the mechanism, and the mechanism-independent one):
an isomerisation A <=> B between species of equal W and enthalpy is a linear
two-state decay, Y_A(t) = Y_eq + (Y_A0 - Y_eq) exp(-lambda t), with lambda
fixed by the rate form (Sec. 2.3 eq. (sourceeq) with the Arrhenius, third-body
and Troe closures).  The same cases pin the oracle in test_oracle.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07094_gb300 as df  # noqa: E402
from paper_2210_07094_gb300 import synth  # noqa: E402

DEV = "cuda:0"
RC = 8.314462618e7  # erg/(mol K)
P_ATM = 101325.0
KC = np.exp(0.7)    # K_c of the isomer pair (a7_B - a7_A = 0.7)


def _run(mech, T, p, Y0, dt, jit, n=40):
    m = df.Mechanism(mech)
    Tt = torch.full((n,), T, dtype=torch.float64, device=DEV)
    pt = torch.full((n,), p, dtype=torch.float64, device=DEV)
    Y = torch.tensor(np.tile(np.array(Y0, float).reshape(3, 1), (1, n)), device=DEV)
    o = df.default_opts()
    o.rtol, o.atol_Y, o.jit = 1e-10, 1e-16, jit
    st, _ = df.integrate(m, Tt, pt, Y, dt, o)
    used, detail = m.jit_info()
    assert int(st.abs().sum()) == 0
    assert used == (jit == 0), detail
    assert torch.max(torch.abs(Tt - T)).item() <= 1e-9  # equal enthalpies: isothermal
    return Y[0].cpu().numpy()


def _expected(Y0, lam, Kc, t):
    ya, yb = Y0[0], Y0[1]
    yeq = (ya + yb) / (1.0 + Kc)
    return yeq + (ya - yeq) * np.exp(-lam * t)


@pytest.mark.parametrize("jit", [0, 1])
def test_third_body_efficiency_on_gpu(jit):
    """A + M <=> B + M with eps_D = 5: lambda = A (1 + 1/K_c) [M] with
    [M] = p/(R T) (Y_A + Y_B + 5 Y_D) (equal molar masses)."""
    T, p = 1300.0, 3 * P_ATM
    mech = synth.isomer_mechanism(kind="three-body", A=4e10, eff={"D": 5.0})
    Y0 = [0.6, 0.1, 0.3]
    Mconc = 10 * p / (RC * T) * (0.6 + 0.1 + 5 * 0.3)
    lam = 4e10 * Mconc * (1 + 1 / KC)
    for frac in (0.5, 2.0):
        ya = _run(mech, T, p, Y0, frac / lam, jit)
        assert np.max(np.abs(ya - _expected(Y0, lam, KC, frac / lam))) <= 1e-8


@pytest.mark.parametrize("jit", [0, 1])
def test_troe_centre_of_falloff_on_gpu(jit):
    """At log10 Pr = 0.4 + 0.67 log10 F_cent the Troe broadening factor is
    exactly F_cent: lambda = k_inf Pr/(1 + Pr) F_cent (1 + 1/K_c)."""
    T, p = 1200.0, 2 * P_ATM
    tr = {"alpha": 0.6, "T3": 200.0, "T1": 1000.0, "T2": 5000.0}
    Fc = (1 - 0.6) * np.exp(-T / 200.0) + 0.6 * np.exp(-T / 1000.0) + np.exp(-5000.0 / T)
    Pr = 10 ** (0.4 + 0.67 * np.log10(Fc))
    Mconc = 10 * p / (RC * T)
    Ainf = 2e5
    mech = synth.isomer_mechanism(kind="falloff-troe", A=Ainf,
                                  low={"A": Pr * Ainf / Mconc, "b": 0.0, "Ea": 0.0}, troe=tr)
    lam = Ainf * Pr / (1 + Pr) * Fc * (1 + 1 / KC)
    Y0 = [0.7, 0.1, 0.2]
    ya = _run(mech, T, p, Y0, 1.0 / lam, jit)
    assert np.max(np.abs(ya - _expected(Y0, lam, KC, 1.0 / lam))) <= 1e-8


@pytest.mark.parametrize("jit", [0, 1])
def test_irreversible_decay_on_gpu(jit):
    """A -> B without the reverse rate: Y_A = Y_A0 exp(-k_f t)."""
    mech = synth.isomer_mechanism(A=5e5, reversible=False)
    for dt in (1e-6, 2e-5):
        ya = _run(mech, 1000.0, P_ATM, [0.5, 0.3, 0.2], dt, jit)
        assert np.max(np.abs(ya - 0.5 * np.exp(-5e5 * dt))) <= 1e-8


@pytest.mark.parametrize("jit", [0, 1])
def test_arrhenius_temperature_dependence_on_gpu(jit):
    """A T^b exp(-Ea/RT) with b and Ea nonzero: lambda = k_f (1 + 1/K_c)."""
    A, b, Ea, T = 1.0e6, 0.7, 50.0, 1500.0
    mech = synth.isomer_mechanism(A=A, b=b, Ea=Ea)
    kf = A * T ** b * np.exp(-Ea * 1e3 / (8.314462618 * T))
    lam = kf * (1 + 1 / KC)
    Y0 = [0.7, 0.1, 0.2]
    ya = _run(mech, T, P_ATM, Y0, 1.0 / lam, jit)
    assert np.max(np.abs(ya - _expected(Y0, lam, KC, 1.0 / lam))) <= 1e-8
