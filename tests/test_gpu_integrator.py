"""GPU parity of the chemistry kernels (rates, Jacobian, integrator) against
the CPU oracle, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07094_gb300 as df  # noqa: E402
from oracle.oracle import Mech  # noqa: E402
from oracle.parity import check_integrator  # noqa: E402
from paper_2210_07094_gb300 import synth  # noqa: E402

DEV = "cuda:0"
TOL_T = 1e-3       # K
TOL_Y = 1e-7       # relative to the largest mass fraction of the cell


def _dev(f):
    return (torch.tensor(f["T"], device=DEV), torch.tensor(f["p"], device=DEV),
            torch.tensor(np.ascontiguousarray(f["Y"]), device=DEV))


@pytest.fixture(scope="module")
def h2():
    mech = synth.h2_air_mechanism()
    return mech, df.Mechanism(mech), Mech(mech)


def _assert_parity(T_in, Y_in, T, Y, To, Yo):
    """Both bars of oracle.parity: the absolute one (TOL_T, TOL_Y) and the error
    relative to the oracle's own change over the step (1e-3 of it), which a
    kernel returning its input fails; the state must have moved."""
    stats = check_integrator(T_in, Y_in, T, Y, To, Yo, tol_T=TOL_T, tol_Y=TOL_Y)
    print(stats)


def test_rhs_matches_oracle(h2):
    mech, m, o = h2
    f = synth.field(1, mech, 1000)
    T, p, Y = _dev(f)
    dydt, qdot = df.rhs(m, T, p, Y)
    dydt, qdot = dydt.cpu().numpy(), qdot.cpu().numpy()
    for c in range(0, 1000, 37):
        y = np.concatenate([[f["T"][c]], f["Y"][:, c]])
        fo, qo = o.rhs(f["p"][c], y)
        scale = np.abs(fo).max()
        assert np.max(np.abs(dydt[:, c] - fo)) <= 1e-12 * scale
        assert abs(qdot[c] - qo) <= 1e-12 * abs(qo) + 1e-300


def test_jacobian_matches_oracle(h2):
    mech, m, o = h2
    f = synth.field(1, mech, 300)
    T, p, Y = _dev(f)
    J = df.jacobian(m, T, p, Y).cpu().numpy()
    for c in range(0, 300, 23):
        y = np.concatenate([[f["T"][c]], f["Y"][:, c]])
        Jo = o.jac(f["p"][c], y)
        scale = np.abs(Jo).max(axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(J[c] - Jo) / scale) <= 1e-10


@pytest.mark.parametrize("method", [0, 1])
def test_integrate_cfg0_all_cells(h2, method):
    """Every cell of a 1000-cell slice of the 0D H2/air field (several blocks and
    a ragged tail)."""
    mech, m, o = h2
    f = synth.field(0, mech, 1000)
    T, p, Y = _dev(f)
    opts = df.default_opts()
    opts.method = method
    status, nsub = df.integrate(m, T, p, Y, f["dt"], opts)
    To, Yo, so, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"])
    assert np.all(so == 0)
    assert int(status.abs().sum()) == 0
    assert int(nsub.min()) >= 1
    _assert_parity(f["T"], f["Y"], T.cpu().numpy(), Y.cpu().numpy(), To, Yo)


def test_integrate_bimodal_full_size_sampled(h2):
    """2^20-cell bimodal field in one persistent launch; 192 sampled cells checked
    against the oracle, all statuses OK, uneven work per cell."""
    mech, m, o = h2
    f = synth.field(1, mech)
    T, p, Y = _dev(f)
    status, nsub = df.integrate(m, T, p, Y, f["dt"])
    st = status.cpu().numpy()
    ns = nsub.cpu().numpy()
    assert np.all(st == 0)
    assert ns.max() >= 3 * ns.min()
    idx = np.random.default_rng(5).choice(f["T"].shape[0], 192, replace=False)
    To, Yo, so, _ = o.integrate(f["T"][idx], f["p"][idx], f["Y"][:, idx], f["dt"])
    assert np.all(so == 0)
    _assert_parity(f["T"][idx], f["Y"][:, idx], T.cpu().numpy()[idx], Y.cpu().numpy()[:, idx], To, Yo)


@pytest.mark.parametrize("n", [1, 31, 33, 97])
def test_small_and_ragged_counts(h2, n):
    mech, m, o = h2
    f = synth.field(1, mech, n)
    T, p, Y = _dev(f)
    status, _ = df.integrate(m, T, p, Y, f["dt"])
    To, Yo, so, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"])
    assert int(status.abs().sum()) == 0
    _assert_parity(f["T"], f["Y"], T.cpu().numpy(), Y.cpu().numpy(), To, Yo)


def test_zero_cells_is_noop(h2):
    _, m, _ = h2
    e = torch.empty(0, dtype=torch.float64, device=DEV)
    df.integrate(m, e, e, torch.empty(0, dtype=torch.float64, device=DEV), 1e-6)


def test_bad_cells_get_status_and_keep_state(h2):
    mech, m, _ = h2
    f = synth.field(0, mech, 64)
    f["T"][3] = np.nan
    f["T"][7] = -100.0
    f["Y"][2, 11] = np.inf
    f["p"][13] = 0.0
    T, p, Y = _dev(f)
    T0, Y0 = T.clone(), Y.clone()
    status, _ = df.integrate(m, T, p, Y, f["dt"])
    st = status.cpu().numpy()
    bad = [3, 7, 11, 13]
    assert np.all(st[bad] == df._lib.CELL_NONFINITE)
    assert np.all(np.delete(st, bad) == 0)
    assert torch.equal(T[bad].nan_to_num(), T0[bad].nan_to_num())
    assert torch.equal(Y[:, bad].nan_to_num(), Y0[:, bad].nan_to_num())


def test_max_substeps_is_reported(h2):
    mech, m, _ = h2
    f = synth.field(1, mech, 128)
    T, p, Y = _dev(f)
    opts = df.default_opts()
    opts.max_substeps = 2
    opts.h0 = 1e-12
    status, nsub = df.integrate(m, T, p, Y, f["dt"], opts)
    assert np.all(status.cpu().numpy() == df._lib.CELL_MAXSTEPS)


def test_zero_rate_mechanism_is_identity_bitwise(h2):
    mech, _, _ = h2
    z = df.Mechanism(synth.zero_rate(mech))
    f = synth.field(0, mech, 256)
    T, p, Y = _dev(f)
    T0, Y0 = T.clone(), Y.clone()
    status, _ = df.integrate(z, T, p, Y, f["dt"])
    assert int(status.abs().sum()) == 0
    assert torch.equal(T, T0) and torch.equal(Y, Y0)


def test_isomer_closed_form_on_gpu():
    """3-species kernel instantiation against the exact two-state decay."""
    A, T0 = 2e5, 1200.0
    mech = synth.isomer_mechanism(A=A)
    m = df.Mechanism(mech)
    lam = A * (1 + np.exp(-0.7))
    n = 40
    T = torch.full((n,), T0, dtype=torch.float64, device=DEV)
    p = torch.full((n,), 101325.0, dtype=torch.float64, device=DEV)
    Y = torch.tensor(np.tile([[0.7], [0.1], [0.2]], (1, n)), device=DEV)
    opts = df.default_opts()
    opts.rtol = 1e-10
    opts.atol_Y = 1e-16
    status, _ = df.integrate(m, T, p, Y, 2.0 / lam, opts)
    yeq = 0.8 / (1 + np.exp(0.7))
    ya = yeq + (0.7 - yeq) * np.exp(-2.0)
    assert int(status.abs().sum()) == 0
    assert np.max(np.abs(Y[0].cpu().numpy() - ya)) <= 1e-8


def test_set_lnA_matches_scaled_mechanism(h2):
    mech, _, _ = h2
    m = df.Mechanism(mech)
    shift = np.random.default_rng(3).uniform(-1, 1, m.n_reactions)
    lnA = torch.tensor(np.log([r["A"] for r in mech["reactions"]]) + shift, device=DEV)
    m.set_lnA(lnA)
    scaled = synth.zero_rate(mech)
    for r, r0, s in zip(scaled["reactions"], mech["reactions"], shift):
        r["A"] = r0["A"] * np.exp(s)
        if "low" in r:
            r["low"]["A"] = r0["low"]["A"] * np.exp(s)
    o = Mech(scaled)
    f = synth.field(1, mech, 200)
    T, p, Y = _dev(f)
    status, _ = df.integrate(m, T, p, Y, f["dt"])
    To, Yo, so, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"])
    assert int(status.abs().sum()) == 0 and np.all(so == 0)
    _assert_parity(f["T"], f["Y"], T.cpu().numpy(), Y.cpu().numpy(), To, Yo)
    m.set_lnA(None)
    T, p, Y = _dev(f)
    df.integrate(m, T, p, Y, f["dt"])
    To, Yo, _, _ = Mech(mech).integrate(f["T"], f["p"], f["Y"], f["dt"])
    _assert_parity(f["T"], f["Y"], T.cpu().numpy(), Y.cpu().numpy(), To, Yo)


# ---------------------------------------------------------------------------
# warp-per-cell path: the 9-species mechanism forced onto it, and the
# 50-species / 300-reaction mechanism that only it runs
# ---------------------------------------------------------------------------

def test_warp_path_9_species(h2):
    mech, m, o = h2
    f = synth.field(1, mech, 600)
    T, p, Y = _dev(f)
    opts = df.default_opts()
    opts.path = 2
    status, nsub = df.integrate(m, T, p, Y, f["dt"], opts)
    To, Yo, so, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"])
    assert int(status.abs().sum()) == 0
    _assert_parity(f["T"], f["Y"], T.cpu().numpy(), Y.cpu().numpy(), To, Yo)
    # same method, same cell: the two paths agree far inside the tolerance
    T2, p2, Y2 = _dev(f)
    opts.path = 1
    df.integrate(m, T2, p2, Y2, f["dt"], opts)
    assert torch.max(torch.abs(T2 - T)).item() <= 1e-6
    assert torch.max(torch.abs(Y2 - Y)).item() <= 1e-10


@pytest.fixture(scope="module")
def chon():
    mech = synth.hydrocarbon_mechanism()
    return mech, df.Mechanism(mech), Mech(mech)


def test_chon_rhs_and_jacobian(chon):
    mech, m, o = chon
    f = synth.field(2, mech, 70)
    T, p, Y = _dev(f)
    dydt, qdot = df.rhs(m, T, p, Y)
    J = df.jacobian(m, T, p, Y).cpu().numpy()
    dydt = dydt.cpu().numpy()
    for c in range(0, 70, 9):
        y = np.concatenate([[f["T"][c]], f["Y"][:, c]])
        fo, _ = o.rhs(f["p"][c], y)
        assert np.max(np.abs(dydt[:, c] - fo)) <= 1e-12 * np.abs(fo).max()
        Jo = o.jac(f["p"][c], y)
        scale = np.abs(Jo).max(axis=1, keepdims=True) + 1e-300
        # some rows of the 300-reaction Jacobian are small remainders of large
        # cancelling reaction terms: 1-ulp rate differences reach 1e-9 of the row
        assert np.max(np.abs(J[c] - Jo) / scale) <= 1e-8
        assert np.linalg.norm(J[c] - Jo) <= 1e-12 * np.linalg.norm(Jo)


def test_chon_integrate_small_all_cells(chon):
    mech, m, o = chon
    f = synth.field(2, mech, 45)
    T, p, Y = _dev(f)
    status, _ = df.integrate(m, T, p, Y, f["dt"])
    To, Yo, so, _ = o.integrate(f["T"], f["p"], f["Y"], f["dt"])
    assert int(status.abs().sum()) == 0 and np.all(so == 0)
    _assert_parity(f["T"], f["Y"], T.cpu().numpy(), Y.cpu().numpy(), To, Yo)


def test_chon_integrate_full_size_sampled(chon):
    """262144 cells of the 50-species field in one launch; 32 sampled cells
    against the oracle."""
    mech, m, o = chon
    f = synth.field(2, mech)
    T, p, Y = _dev(f)
    status, nsub = df.integrate(m, T, p, Y, f["dt"])
    assert int(status.abs().sum()) == 0
    idx = np.random.default_rng(11).choice(f["T"].shape[0], 32, replace=False)
    To, Yo, so, _ = o.integrate(f["T"][idx], f["p"][idx], f["Y"][:, idx], f["dt"])
    assert np.all(so == 0)
    _assert_parity(f["T"][idx], f["Y"][:, idx], T.cpu().numpy()[idx], Y.cpu().numpy()[:, idx], To, Yo)
