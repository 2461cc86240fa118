"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a closed-form solution of a
reduced problem, an invariant of the exact ODE, the equilibrium state found by
an independent method (element-potential Gibbs minimisation), the derivative
definition (finite differences), or the published order of a method.
"""
import numpy as np
import pytest
from scipy import integrate, optimize

from oracle.oracle import Mech
from paper_2210_07094_gb300 import synth

R = 8.314462618
RC = 8.314462618e7  # erg/(mol K)
P_ATM = 101325.0


@pytest.fixture(scope="module")
def h2():
    return Mech(synth.h2_air_mechanism())


@pytest.fixture(scope="module")
def chon():
    return Mech(synth.hydrocarbon_mechanism())


# ---------------------------------------------------------------------------
# thermo (NASA-7, one range)
# ---------------------------------------------------------------------------

def test_enthalpy_and_entropy_are_integrals_of_cp(h2, chon):
    """H(T2) - H(T1) = int cp dT and S(T2) - S(T1) = int cp/T dT (quadrature)."""
    for m in (h2, chon):
        for k in range(0, m.N, max(1, m.N // 9)):
            cp = lambda T: m.thermo(T)[0][k]
            for T1, T2 in ((300.0, 1200.0), (900.0, 2900.0)):
                dH = integrate.quad(cp, T1, T2, epsabs=0, epsrel=1e-13)[0]
                dS = integrate.quad(lambda T: cp(T) / T, T1, T2, epsabs=0, epsrel=1e-13)[0]
                _, h1, s1 = m.thermo(T1)
                _, h2_, s2 = m.thermo(T2)
                assert abs((h2_[k] * T2 - h1[k] * T1) - dH) <= 1e-10 * abs(dH)
                assert abs((s2[k] - s1[k]) - dS) <= 1e-10 * abs(dS)


def test_reference_state_matches_drawn_formation_data(h2, chon):
    """H(298.15 K) equals the drawn heat of formation; S(298.15)/R the drawn entropy."""
    for m in (h2, chon):
        _, h, s = m.thermo(298.15)
        for k, sp in enumerate(m.json["species"]):
            assert abs(h[k] * R * 298.15 / 1e3 - sp["Hf298"]) <= 1e-9 * max(1.0, abs(sp["Hf298"]))
            assert abs(s[k] - sp["S298_R"]) <= 1e-12 * sp["S298_R"]


def test_gibbs_helmholtz(h2):
    """d(g/RT)/dT = -h/(R T^2) (thermodynamic identity; central difference)."""
    for T in (700.0, 1500.0, 2600.0):
        dT = 1e-3
        _, hp, sp = h2.thermo(T + dT)
        _, hm, sm = h2.thermo(T - dT)
        _, h0, _ = h2.thermo(T)
        dg = ((hp - sp) - (hm - sm)) / (2 * dT)
        assert np.allclose(dg, -h0 / T, rtol=1e-7, atol=0)


# ---------------------------------------------------------------------------
# rates through closed-form isomerisation problems (A <=> B, dT/dt = 0)
# ---------------------------------------------------------------------------

def _iso_run(mech, T, p, Y0, dt, rtol=1e-12):
    m = Mech(mech)
    T1, Y1, st, _ = m.integrate(np.array([T]), np.array([p]), np.array(Y0, float).reshape(3, 1),
                                dt, rtol=rtol, atolY=1e-22, atolT=1e-12)
    assert st[0] == 0
    return m, T1[0], Y1[:, 0]


def _iso_expected(Y0, lam, Kc, t):
    ya, yb = Y0[0], Y0[1]
    yeq = (ya + yb) / (1.0 + Kc)  # k_r/(k_f+k_r) = 1/(1+Kc)
    return yeq + (ya - yeq) * np.exp(-lam * t)


@pytest.mark.parametrize("A,b,Ea,T", [(2.0e5, 0.0, 0.0, 1200.0), (1.0e6, 0.7, 50.0, 1500.0),
                                      (3.0e4, -1.2, 120.0, 2400.0)])
def test_isomerisation_closed_form(A, b, Ea, T):
    """Y_A(t) = Y_eq + (Y_A0 - Y_eq) exp(-(k_f + k_r) t) with the Arrhenius k_f and
    k_r = k_f / K_c, K_c = exp(-dg/RT) = exp(a7_B - a7_A) for equal-enthalpy isomers."""
    a7b = 10.7
    mech = synth.isomer_mechanism(A=A, b=b, Ea=Ea, a7_b=a7b)
    kf = A * T ** b * np.exp(-Ea * 1e3 / (R * T))
    Kc = np.exp(a7b - 10.0)
    lam = kf * (1.0 + 1.0 / Kc)
    Y0 = [0.7, 0.1, 0.2]
    for frac in (0.3, 1.0, 3.0):
        dt = frac / lam
        m, T1, Y1 = _iso_run(mech, T, P_ATM, Y0, dt)
        assert T1 == pytest.approx(T, abs=1e-9)
        ya = _iso_expected(Y0, lam, Kc, dt)
        assert abs(Y1[0] - ya) <= 1e-11
        assert abs(Y1[0] + Y1[1] - 0.8) <= 1e-14
        assert Y1[2] == 0.2


def test_irreversible_decay():
    """Irreversible A -> B: Y_A = Y_A0 exp(-k_f t)."""
    mech = synth.isomer_mechanism(A=5e5, reversible=False)
    for dt in (1e-6, 4e-6, 2e-5):
        _, _, Y1 = _iso_run(mech, 1000.0, P_ATM, [0.5, 0.3, 0.2], dt)
        assert abs(Y1[0] - 0.5 * np.exp(-5e5 * dt)) <= 1e-11


def test_third_body_efficiencies():
    """A + M <=> B + M with eps_D = 5: decay rate (k_f + k_r) [M],
    [M] = p/(R T) (Y_A + Y_B + 5 Y_D) for species of equal W."""
    T, p = 1300.0, 3 * P_ATM
    mech = synth.isomer_mechanism(kind="three-body", A=4e10, eff={"D": 5.0})
    Y0 = [0.6, 0.1, 0.3]
    Mconc = 10 * p / (RC * T) * (0.6 + 0.1 + 5 * 0.3)
    Kc = np.exp(0.7)
    lam = 4e10 * Mconc * (1 + 1 / Kc)
    for frac in (0.5, 2.0):
        _, _, Y1 = _iso_run(mech, T, p, Y0, frac / lam)
        assert abs(Y1[0] - _iso_expected(Y0, lam, Kc, frac / lam)) <= 1e-11


@pytest.mark.parametrize("Pr", [1.0, 9.0, 0.05])
def test_troe_reduces_to_lindemann(Pr):
    """With F_cent = 1 (T***, T*, T** -> infinity) the Troe form is the Lindemann
    form k = k_inf Pr / (1 + Pr)."""
    T, p = 1200.0, P_ATM
    Mconc = 10 * p / (RC * T)  # all efficiencies 1
    Ainf = 3e5
    A0 = Pr * Ainf / Mconc
    mech = synth.isomer_mechanism(kind="falloff-troe", A=Ainf, low={"A": A0, "b": 0.0, "Ea": 0.0},
                                  troe={"alpha": 0.5, "T3": 1e300, "T1": 1e300, "T2": 1e300})
    Kc = np.exp(0.7)
    lam = Ainf * Pr / (1 + Pr) * (1 + 1 / Kc)
    Y0 = [0.7, 0.1, 0.2]
    _, _, Y1 = _iso_run(mech, T, p, Y0, 1.0 / lam)
    assert abs(Y1[0] - _iso_expected(Y0, lam, Kc, 1.0 / lam)) <= 1e-11


def test_troe_centre_of_falloff():
    """At log10 Pr = -c = 0.4 + 0.67 log10 F_cent the broadening factor is exactly
    F_cent (the Troe interpolation term vanishes), so k = k_inf Pr/(1+Pr) F_cent
    with F_cent = (1-a) exp(-T/T***) + a exp(-T/T*) + exp(-T**/T)."""
    T, p = 1200.0, 2 * P_ATM
    tr = {"alpha": 0.6, "T3": 200.0, "T1": 1000.0, "T2": 5000.0}
    Fc = (1 - 0.6) * np.exp(-T / 200.0) + 0.6 * np.exp(-T / 1000.0) + np.exp(-5000.0 / T)
    Pr = 10 ** (0.4 + 0.67 * np.log10(Fc))
    Mconc = 10 * p / (RC * T)
    Ainf = 2e5
    mech = synth.isomer_mechanism(kind="falloff-troe", A=Ainf,
                                  low={"A": Pr * Ainf / Mconc, "b": 0.0, "Ea": 0.0}, troe=tr)
    Kc = np.exp(0.7)
    lam = Ainf * Pr / (1 + Pr) * Fc * (1 + 1 / Kc)
    Y0 = [0.7, 0.1, 0.2]
    _, _, Y1 = _iso_run(mech, T, p, Y0, 1.0 / lam)
    assert abs(Y1[0] - _iso_expected(Y0, lam, Kc, 1.0 / lam)) <= 1e-11


# ---------------------------------------------------------------------------
# integrator invariants on the seeded workloads
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg1_run(h2):
    f = synth.field(1, h2.json, 96)
    T1, Y1, st, ns = h2.integrate(f["T"], f["p"], f["Y"], f["dt"])
    return f, T1, Y1, st, ns


def test_all_cells_converge(cfg1_run):
    _, _, _, st, ns = cfg1_run
    assert np.all(st == 0)
    assert ns.max() >= 3 * ns.min()  # the bimodal field has uneven stiffness


def test_element_and_mass_conservation(h2, cfg1_run):
    """Linear invariants of the exact ODE: element moles and sum(Y)."""
    f, T1, Y1, _, _ = cfg1_run
    e0 = h2.elem @ (f["Y"] / h2.W[:, None])
    e1 = h2.elem @ (Y1 / h2.W[:, None])
    assert np.max(np.abs(e1 - e0) / np.abs(e0).max(axis=0)) <= 1e-12
    assert np.max(np.abs(Y1.sum(axis=0) - f["Y"].sum(axis=0))) <= 1e-12


def test_enthalpy_conservation(h2, cfg1_run):
    """Adiabatic constant-pressure reactor: h(T, Y) is constant."""
    f, T1, Y1, _, _ = cfg1_run
    for c in range(0, T1.shape[0], 7):
        h0 = h2.enthalpy_mass(f["T"][c], f["Y"][:, c])
        h1 = h2.enthalpy_mass(T1[c], Y1[:, c])
        cp_scale = 1.5e3 * f["T"][c]  # ~cp T in J/kg
        assert abs(h1 - h0) <= 1e-9 * cp_scale


def test_zero_rate_mechanism_is_identity(h2):
    z = Mech(synth.zero_rate(h2.json))
    f = synth.field(0, h2.json, 32)
    T1, Y1, st, _ = z.integrate(f["T"], f["p"], f["Y"], f["dt"])
    assert np.all(st == 0)
    assert np.array_equal(T1, f["T"]) and np.array_equal(Y1, f["Y"])


def test_self_convergence_and_time_additivity(h2):
    """rtol 1e-10 vs 1e-12 and one call over dt vs two over dt/2 agree far inside
    the GPU tolerance (1e-3 K, 1e-7 max Y)."""
    f = synth.field(1, h2.json, 24)
    Ta, Ya, _, _ = h2.integrate(f["T"], f["p"], f["Y"], f["dt"], rtol=1e-10)
    Tb, Yb, _, _ = h2.integrate(f["T"], f["p"], f["Y"], f["dt"], rtol=1e-12, atolT=1e-12,
                                atolY=1e-22)
    Th, Yh, _, _ = h2.integrate(f["T"], f["p"], f["Y"], f["dt"] / 2)
    Th, Yh, _, _ = h2.integrate(Th, f["p"], Yh, f["dt"] / 2)
    for T, Y in ((Ta, Ya), (Th, Yh)):
        assert np.max(np.abs(T - Tb)) <= 1e-6
        assert np.max(np.abs(Y - Yb) / Yb.max(axis=0)) <= 1e-10


def _element_potential_equilibrium(m, T, p, b):
    """Gibbs minimum at (T, p) for element moles b [mol/g], by element potentials:
    n_k = N exp(-g_k/RT - ln(p/p0) + sum_e lam_e a_ek)."""
    _, h, s = m.thermo(T)
    mu0 = h - s + np.log(p / P_ATM)
    A = m.elem
    ne = A.shape[0]

    def resid(x):
        lam, lnN = x[:ne], x[ne]
        n = np.exp(lnN - mu0 + A.T @ lam)
        return np.concatenate([(A @ n - b) / b, [(n.sum() - np.exp(lnN)) / np.exp(lnN)]])

    n_guess = np.full(m.N, b.sum() / m.N)
    x0 = np.concatenate([np.zeros(ne), [np.log(n_guess.sum())]])
    # least-squares start: lam from the largest species
    sol = optimize.root(resid, x0, method="lm", options={"xtol": 1e-15, "ftol": 1e-15,
                                                         "maxiter": 20000})
    lam, lnN = sol.x[:ne], sol.x[ne]
    n = np.exp(lnN - mu0 + A.T @ lam)
    assert np.max(np.abs(resid(sol.x))) < 1e-10
    return n / n.sum()


def test_long_time_equilibrium(h2):
    """After a long integration the state satisfies detailed balance reaction by
    reaction, and its composition equals the Gibbs minimum found by element
    potentials at the same T, p and element amounts."""
    nu = h2.nu
    assert np.linalg.matrix_rank(nu) == h2.N - np.linalg.matrix_rank(h2.elem)
    f = synth.field(0, h2.json, 1)
    T0 = np.array([2200.0])
    T1, Y1, st, _ = h2.integrate(T0, f["p"], f["Y"], 1e4, rtol=1e-10, atolY=1e-25)
    assert st[0] == 0
    r = h2.rates(T1[0], f["p"][0], Y1[:, 0])
    C = r["rho"] * Y1[:, 0] / h2.W
    for j in range(h2.M):
        qf = r["kf"][j] * np.prod(C[h2.reac[j, :h2.nreac[j]]])
        qr = r["kr"][j] * np.prod(C[h2.prod[j, :h2.nprod[j]]])
        assert abs(qf - qr) <= 1e-6 * max(qf, qr)
    b = h2.elem @ (Y1[:, 0] / h2.W)
    X_eq = _element_potential_equilibrium(h2, T1[0], f["p"][0], b)
    X = (Y1[:, 0] / h2.W) / np.sum(Y1[:, 0] / h2.W)
    big = X_eq > 1e-12
    assert np.max(np.abs(X[big] - X_eq[big]) / X_eq[big]) <= 1e-6


# ---------------------------------------------------------------------------
# Jacobian (complex step) against central finite differences
# ---------------------------------------------------------------------------

def _fd_jac(m, p, y):
    """Central differences with one Richardson extrapolation (O(h^4))."""
    n = y.shape[0]
    J = np.zeros((n, n))

    def central(j, hs):
        yp, ym = y.copy(), y.copy()
        yp[j] += hs
        ym[j] -= hs
        return (m.rhs(p, yp)[0] - m.rhs(p, ym)[0]) / (2 * hs)

    for j in range(n):
        hs = 0.5 if j == 0 else 1e-4 * max(abs(y[j]), 1e-2)
        J[:, j] = (4 * central(j, hs / 2) - central(j, hs)) / 3
    return J


def test_jacobian_vs_finite_differences(h2, chon):
    for m, cfg, ncell in ((h2, 1, 6), (chon, 2, 2)):
        f = synth.field(cfg, m.json, ncell)
        for c in range(ncell):
            y = np.concatenate([[f["T"][c]], f["Y"][:, c]])
            J = m.jac(f["p"][c], y)
            Jf = _fd_jac(m, f["p"][c], y)
            scale = np.abs(Jf).max(axis=1, keepdims=True) + 1e-300
            assert np.max(np.abs(J - Jf) / scale) <= 1e-7


# ---------------------------------------------------------------------------
# RODAS4 replay (reference for the discrete adjoint)
# ---------------------------------------------------------------------------

def _hot_state(h2):
    f = synth.field(1, h2.json, 64)
    c = int(np.argmax(f["T"]))
    return f["p"][c], np.concatenate([[f["T"][c]], f["Y"][:, c]])


def test_rodas4_convergence_order(h2):
    """Global error of the fixed-step replay falls as h^4 (RODAS4 has order 4)."""
    p, y0 = _hot_state(h2)
    H = 2e-7
    Tr, Yr, st, _ = h2.integrate(np.array([y0[0]]), np.array([p]), y0[1:].reshape(-1, 1), H,
                                 rtol=1e-13, atolY=1e-24, atolT=1e-12)
    yref = np.concatenate([Tr, Yr[:, 0]])
    errs = []
    for n in (4, 8, 16):
        y = h2.ros_replay(p, y0, np.full(n, H / n))
        errs.append(np.max(np.abs(y - yref) / (np.abs(yref) + 1e-12)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 10.0 < r1 < 26.0 and 10.0 < r2 < 26.0, errs


def test_rodas4_stiff_decay(h2):
    """L-stable: one step of length h on the linear isomer problem with
    z = h (k_f + k_r) -> infinity lands on the equilibrium Y_eq = (Y_A + Y_B)/(1 + K_c)
    with an error that falls like 1/z (R(z) -> 0)."""
    m = Mech(synth.isomer_mechanism(A=2e5))
    y0 = np.array([1200.0, 0.7, 0.1, 0.2])
    lam = 2e5 * (1 + np.exp(-0.7))
    yeq = 0.8 / (1 + np.exp(0.7))
    e = [m.ros_replay(P_ATM, y0, np.array([z / lam]))[1] - yeq for z in (1e5, 1e7)]
    assert abs(e[1]) <= 1e-6
    assert 80.0 < e[0] / e[1] < 120.0


def test_rodas4_embedded_error_order(h2):
    """The embedded estimate is O(h^4) per step (third-order companion)."""
    p, y0 = _hot_state(h2)
    e = [np.max(np.abs(h2.ros_step(p, y0, h)[1][1:])) for h in (4e-8, 2e-8)]
    assert 10.0 < e[0] / e[1] < 26.0, e


def test_replay_directional_derivative_vs_fd(h2):
    """Complex-step derivative of the replayed map equals central differences."""
    p, y0 = _hot_state(h2)
    hs = np.full(6, 3e-8)
    rng = np.random.default_rng(1)
    dlnA = rng.standard_normal(h2.M)
    dy0 = np.zeros_like(y0)
    dy0[0] = 1.0
    wY = rng.standard_normal(h2.N)
    for kw in ({"dy0": dy0}, {"dlnA": dlnA}):
        d_cs = h2.ros_replay_dir(p, y0, hs, wT=1.0, wY=wY, wQ=1e-9, **kw)

        def L(sign):
            mm = Mech(h2.json)
            if "dlnA" in kw:
                mm.A *= np.exp(sign * eps * dlnA)
                mm.A0 *= np.exp(sign * eps * dlnA)
                yy = y0
            else:
                yy = y0 + sign * eps * dy0
            y = mm.ros_replay(p, yy, hs)
            fq = mm.rhs(p, y)[1]
            return y[0] + wY @ y[1:] + 1e-9 * fq

        d = []
        for eps in (1e-2, 5e-3) if "dy0" in kw else (2e-3, 1e-3):
            d.append((L(1) - L(-1)) / (2 * eps))
        d_fd = (4 * d[1] - d[0]) / 3  # Richardson
        assert abs(d_cs - d_fd) <= 1e-6 * abs(d_fd), (d_cs, d_fd)


def test_ignition_helper_zero_rate_and_additivity():
    """The oracle's multi-step helper: with every rate zero nothing moves and
    the largest dT/dt (0) is found at t = 0; otherwise its final state is the
    single integration over the whole window (time additivity)."""
    mech = synth.h2_air_mechanism()
    f = synth.field(0, mech, 6, seed=3)
    z = Mech(synth.zero_rate(mech))
    T, Y, tb, best = z.ignition(f["T"], f["p"], f["Y"], 1e-6, 3, grid=2)
    assert np.array_equal(T, f["T"]) and np.array_equal(Y, f["Y"])
    assert np.all(tb == 0.0) and np.all(best == 0.0)
    o = Mech(mech)
    T1, Y1, tb1, best1 = o.ignition(f["T"], f["p"], f["Y"], 2e-6, 3, grid=2)
    T2, Y2, _, _ = o.integrate(f["T"], f["p"], f["Y"], 6e-6)
    assert np.max(np.abs(T1 - T2)) <= 1e-7
    assert np.max(np.abs(Y1 - Y2)) <= 1e-11
    assert np.all((tb1 >= 0.0) & (tb1 < 6e-6)) and np.all(np.isfinite(best1))


# ---------------------------------------------------------------------------
# constant-volume reactor (Sec. 2.2: df0DFoam's constant-volume case)
# ---------------------------------------------------------------------------

def test_constant_volume_isomerisation_closed_form():
    """Equal-enthalpy isomers release no heat, so at constant volume as at
    constant pressure T stays fixed and Y_A relaxes with rate k_f + k_r."""
    A, b, Ea, T, a7b = 1.0e6, 0.7, 50.0, 1500.0, 10.7
    mech = synth.isomer_mechanism(A=A, b=b, Ea=Ea, a7_b=a7b)
    kf = A * T ** b * np.exp(-Ea * 1e3 / (R * T))
    Kc = np.exp(a7b - 10.0)
    lam = kf * (1.0 + 1.0 / Kc)
    m = Mech(mech)
    Y0 = [0.7, 0.1, 0.2]
    for frac in (0.3, 1.0, 3.0):
        dt = frac / lam
        T1, Y1, st, _ = m.integrate(np.array([T]), np.array([P_ATM]), np.array(Y0, float).reshape(3, 1), dt,
                                    rtol=1e-12, atolY=1e-22, atolT=1e-12, constant_volume=True)
        assert st[0] == 0
        assert T1[0] == pytest.approx(T, abs=1e-9)
        assert abs(Y1[0, 0] - _iso_expected(Y0, lam, Kc, dt)) <= 1e-11


def test_constant_volume_conserves_internal_energy_and_heats_more(h2):
    """u(T, Y) is conserved at constant volume; the same composition change
    releases the same heat into cv instead of cp, so T rises more, by about
    cp/cv for a small change."""
    f = synth.field(1, h2.json, 24, seed=41)
    Tv, Yv, sv, _ = h2.integrate(f["T"], f["p"], f["Y"], f["dt"], constant_volume=True)
    Tp, Yp, sp, _ = h2.integrate(f["T"], f["p"], f["Y"], f["dt"])
    assert np.all(sv == 0) and np.all(sp == 0)
    for c in range(24):
        u0 = h2.internal_energy_mass(f["T"][c], f["Y"][:, c])
        u1 = h2.internal_energy_mass(Tv[c], Yv[:, c])
        assert abs(u1 - u0) <= 1e-9 * 1.5e3 * f["T"][c]
    dTp, dTv = Tp - f["T"], Tv - f["T"]
    big = np.abs(dTp) > 1e-3
    assert big.sum() >= 4
    ratio = dTv[big] / dTp[big]
    assert np.all((ratio > 1.1) & (ratio < 1.6)), ratio  # cp/cv of air-like mixtures ~1.3-1.4


def test_constant_volume_jacobian_vs_finite_differences(h2):
    f = synth.field(1, h2.json, 4, seed=5)
    for c in range(4):
        y = np.concatenate([[f["T"][c]], f["Y"][:, c]])
        rho = h2.density(f["T"][c], f["p"][c], f["Y"][:, c])
        J = h2.jac_v(rho, y)
        n = y.shape[0]
        Jf = np.zeros((n, n))
        for j in range(n):
            hs = 0.5 if j == 0 else 1e-4 * max(abs(y[j]), 1e-2)
            cols = []
            for hh in (hs, hs / 2):
                yp, ym = y.copy(), y.copy()
                yp[j] += hh
                ym[j] -= hh
                cols.append((h2.rhs_v(rho, yp)[0] - h2.rhs_v(rho, ym)[0]) / (2 * hh))
            Jf[:, j] = (4 * cols[1] - cols[0]) / 3
        scale = np.abs(Jf).max(axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(J - Jf) / scale) <= 1e-7
        # the constant-volume right-hand side differs from the constant-pressure one
        # only through rho (same here) and cv, U in the temperature row
        fv = h2.rhs_v(rho, y)[0]
        fp = h2.rhs(f["p"][c], y)[0]
        assert np.allclose(fv[1:], fp[1:], rtol=1e-12, atol=0)


def test_parity_check_rejects_a_kernel_that_returns_its_input():
    """The acceptance check used by every integrator parity test must fail a
    'kernel' that returns its input unchanged, on the 0D H2/air field where
    the whole change over dt is below the absolute bar (1e-3 K, 1e-7 max Y),
    and one that takes a slightly wrong step (dt * (1 - 1e-2)); the oracle's
    own result at a tighter tolerance passes."""
    from oracle.parity import check_integrator
    mech = synth.h2_air_mechanism()
    o = Mech(mech)
    f = synth.field(0, mech, 300)
    To, Yo, so, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"])
    assert np.all(so == 0)
    # the absolute bar alone cannot tell: the whole change is below it
    assert np.abs(To - f["T"]).max() < 1e-3
    assert (np.abs(Yo - f["Y"]).max(axis=0) / Yo.max(axis=0)).max() < 1e-7
    with pytest.raises(AssertionError):
        check_integrator(f["T"], f["Y"], f["T"], f["Y"], To, Yo)
    Tw, Yw, _, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"] * (1 - 1e-2))
    with pytest.raises(AssertionError):
        check_integrator(f["T"], f["Y"], Tw, Yw, To, Yo)
    Tt, Yt, _, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"], rtol=1e-12, atolT=1e-12)
    check_integrator(f["T"], f["Y"], Tt, Yt, To, Yo)


def test_ignition_time_of_the_logistic_closed_form():
    """A + B -> 2 B with equal molar masses and heat capacities and a small heat
    of reaction: dY_B/dt = r Y_A Y_B with r = A rho / W, a logistic curve whose
    rate -- and dT/dt with it -- peaks when Y_A = Y_B, at
    t* = ln(Y_A0 / Y_B0) / (r (Y_A0 + Y_B0)).  The oracle's time of the largest
    dT/dt (Sec. 4.1's ignition delay) on a grid of dt/16 lies within half a grid
    spacing of t*, plus the shift from the 0.1 K the mixture heats (rho moves by
    1e-4)."""
    mech = synth.autocatalytic_mechanism()
    o = Mech(mech)
    YA = np.array([0.5, 0.5, 0.3, 0.6])
    YB = np.array([1e-3, 1e-4, 1e-3, 5e-3])
    Y = np.vstack([YA, YB, 1.0 - YA - YB])
    T0, p = np.full(4, 1000.0), np.full(4, 101325.0)
    rho = 10 * 101325.0 * 30.0 / (8.314462618e7 * 1000.0)  # g/cm^3, cgs gas constant
    tstar = np.log(YA / YB) / (1e7 * rho / 30.0 * (YA + YB))
    dt, grid = 0.01, 16
    _, _, tig, _ = o.ignition(T0, p, Y, dt, 25, grid=grid)
    assert np.all(np.abs(tig - tstar) <= 0.5 * dt / grid + 1e-3 * tstar), (tig, tstar)
