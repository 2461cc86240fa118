"""GPU discrete adjoint against (a) the oracle's complex-step derivative of the
same discrete map (RODAS4 replayed with the GPU's accepted step sequence, read
from the checkpoints) and (b) central finite differences of that map."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07094_gb300 as df  # noqa: E402
from oracle.oracle import Mech  # noqa: E402
from paper_2210_07094_gb300 import synth  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def setup():
    mech = synth.h2_air_mechanism()
    return mech, df.Mechanism(mech), Mech(mech)


def _dev(f):
    return (torch.tensor(f["T"], device=DEV), torch.tensor(f["p"], device=DEV),
            torch.tensor(np.ascontiguousarray(f["Y"]), device=DEV))


def _run(setup, cfg, ncells, seed, opts=None):
    mech, m, o = setup
    f = synth.field(cfg, mech, ncells, seed=seed)
    T, p, Y = _dev(f)
    N = m.n_species
    rng = np.random.default_rng(seed)
    gT = rng.standard_normal(ncells)
    gY = rng.standard_normal((N, ncells))
    gQ = rng.standard_normal(ncells) * 1e-9
    r = df.adjoint(m, T, p, Y, f["dt"], torch.tensor(gT, device=DEV), torch.tensor(gY, device=DEV),
                   torch.tensor(gQ, device=DEV), opts=opts)
    return f, gT, gY, gQ, r


def _steps(r, N, c, max_steps=64):
    ns = int(r["nsub"][c])
    ck = r["workspace"][: r["nsub"].numel() * max_steps * (N + 2) * 8].view(torch.float64)
    ck = ck.view(-1, max_steps, N + 2)[c, :ns].cpu().numpy()
    return ck[:, -1]


@pytest.mark.parametrize("cfg", [1, 3])
def test_adjoint_matches_oracle_complex_step(setup, cfg):
    mech, m, o = setup
    n = 48
    f, gT, gY, gQ, r = _run(setup, cfg, n, 100 + cfg)
    assert int(r["status"].abs().sum()) == 0
    gT0, gY0, glnA = r["gT0"].cpu().numpy(), r["gY0"].cpu().numpy(), r["g_lnA"].cpu().numpy()
    rng = np.random.default_rng(7)
    dlnA = rng.standard_normal(m.n_reactions)
    tot_gpu_A, tot_or_A = glnA @ dlnA, 0.0
    for c in range(n):
        hs = _steps(r, m.n_species, c)
        y0 = np.concatenate([[f["T"][c]], f["Y"][:, c]])
        dy0 = rng.standard_normal(m.n_species + 1) * np.r_[1.0, np.full(m.n_species, 1e-4)]
        d_or = o.ros_replay_dir(f["p"][c], y0, hs, wT=gT[c], wY=gY[:, c], wQ=gQ[c], dy0=dy0)
        d_gpu = gT0[c] * dy0[0] + gY0[:, c] @ dy0[1:]
        assert abs(d_gpu - d_or) <= 1e-6 * max(abs(d_or), 1e-12), (c, d_gpu, d_or)
        tot_or_A += o.ros_replay_dir(f["p"][c], y0, hs, wT=gT[c], wY=gY[:, c], wQ=gQ[c], dlnA=dlnA)
    assert abs(tot_gpu_A - tot_or_A) <= 1e-6 * abs(tot_or_A)


def test_adjoint_matches_central_differences(setup):
    """Central differences (step 1e-6 relative) of the replayed RODAS4 map."""
    mech, m, o = setup
    n = 8
    f, gT, gY, gQ, r = _run(setup, 1, n, 31)
    gT0, gY0, glnA = r["gT0"].cpu().numpy(), r["gY0"].cpu().numpy(), r["g_lnA"].cpu().numpy()

    def L(c, y0, mm):
        hs = _steps(r, m.n_species, c)
        y = mm.ros_replay(f["p"][c], y0, hs)
        return gT[c] * y[0] + gY[:, c] @ y[1:] + gQ[c] * mm.rhs(f["p"][c], y)[1]

    for c in range(n):
        y0 = np.concatenate([[f["T"][c]], f["Y"][:, c]])
        eps = 1e-6 * y0[0]
        e = np.zeros_like(y0)
        e[0] = eps
        fd = (L(c, y0 + e, o) - L(c, y0 - e, o)) / (2 * eps)
        assert abs(gT0[c] - fd) <= 1e-5 * max(abs(fd), 1e-6 * abs(gT[c])), (c, gT0[c], fd)
    # ln A of the most sensitive reactions, summed over the cells.  The loss
    # weighs Y only: a T term (T ~ 2000 K, rounding ~4e-13 K) would drown a
    # 1e-6 central difference in rounding noise.
    T, p, Y = _dev(f)
    r2 = df.adjoint(m, T, p, Y, f["dt"], gY1=torch.tensor(gY, device=DEV))
    glnA = r2["g_lnA"].cpu().numpy()

    def LY(c, y0, mm):
        hs = _steps(r2, m.n_species, c)
        return gY[:, c] @ mm.ros_replay(f["p"][c], y0, hs)[1:]

    for j in np.argsort(-np.abs(glnA))[:3]:
        eps = 1e-6
        tot = 0.0
        for sgn in (1, -1):
            mm = Mech(mech)
            mm.A[j] *= np.exp(sgn * eps)
            mm.A0[j] *= np.exp(sgn * eps)
            tot += sgn * sum(LY(c, np.concatenate([[f["T"][c]], f["Y"][:, c]]), mm) for c in range(n))
        fd = tot / (2 * eps)
        # rounding noise of the difference: ~ulp(L) * sqrt(cells) / (2 eps) ~ 3e-10
        assert abs(glnA[j] - fd) <= 1e-5 * abs(fd) + 5e-10, (j, glnA[j], fd)


def test_adjoint_deterministic_and_full_size(setup):
    """65536 cells (the adjoint workload, the launch the bench times): all
    cells OK, the gradients bitwise reproducible across calls, and for sampled
    cells every component of (dL/dT0, dL/dY0) against the oracle's
    complex-step derivative of the same replayed RODAS4 map (the ln A gradient
    sums over all cells; its components are checked on single cells above)."""
    mech, m, o = setup
    N = m.n_species
    f = synth.field(3, mech)
    T, p, Y = _dev(f)
    n = T.numel()
    rng = np.random.default_rng(65536)
    gT = rng.standard_normal(n)
    gY = rng.standard_normal((N, n))
    gQ = rng.standard_normal(n) * 1e-9
    args = [torch.tensor(a, device=DEV) for a in (gT, gY, gQ)]
    r1 = df.adjoint(m, T, p, Y, f["dt"], *args)
    r2 = df.adjoint(m, T, p, Y, f["dt"], *args)
    assert int(r1["status"].abs().sum()) == 0
    for k in ("g_lnA", "gT0", "gY0"):
        assert torch.equal(r1[k], r2[k]), k
    assert torch.isfinite(r1["g_lnA"]).all()
    gT0, gY0 = r1["gT0"].cpu().numpy(), r1["gY0"].cpu().numpy()
    for c in (0, 12345, 40000, n - 1):
        hs = _steps(r1, N, c)
        y0 = np.concatenate([[f["T"][c]], f["Y"][:, c]])
        ref = np.array([o.ros_replay_dir(f["p"][c], y0, hs, wT=gT[c], wY=gY[:, c], wQ=gQ[c],
                                         dy0=np.eye(N + 1)[i]) for i in range(N + 1)])
        g = np.r_[gT0[c], gY0[:, c]]
        bound = 1e-6 * np.abs(ref) + 1e-9 * np.abs(ref).max()
        assert np.all(np.abs(g - ref) <= bound), (c, float(np.max(np.abs(g - ref) / bound)))


@pytest.mark.parametrize("cfg,ncells", [(1, 777), (3, 4099)])
def test_stored_stages_match_recompute(setup, cfg, ncells):
    """The reverse sweep reading the forward pass's stored stages and LU
    factors gives bitwise the result of recomputing each step (compact
    workspace), on ragged cell counts; the checkpoints agree too."""
    mech, m, o = setup
    f = synth.field(cfg, mech, ncells, seed=500 + cfg)
    T, p, Y = _dev(f)
    rng = np.random.default_rng(cfg)
    gT = torch.tensor(rng.standard_normal(ncells), device=DEV)
    gY = torch.tensor(rng.standard_normal((m.n_species, ncells)), device=DEV)
    gQ = torch.tensor(rng.standard_normal(ncells) * 1e-9, device=DEV)
    full = df.adjoint(m, T, p, Y, f["dt"], gT, gY, gQ, max_steps=32)
    compact = df.adjoint(m, T, p, Y, f["dt"], gT, gY, gQ, max_steps=32, store_stages=False)
    n_ck = ncells * 32 * (m.n_species + 2) * 8
    assert full["workspace"].numel() > compact["workspace"].numel() >= n_ck
    assert int(full["status"].abs().sum()) == 0
    for k in ("status", "nsub", "gT0", "gY0", "g_lnA"):
        assert torch.equal(full[k], compact[k]), k
    # checkpoint slots past a cell's accepted steps are never written
    used = torch.arange(32, device=DEV)[None, :] < full["nsub"][:, None]
    ck_f, ck_c = (r["workspace"][:n_ck].view(torch.float64).view(ncells, 32, -1) for r in (full, compact))
    assert torch.equal(ck_f[used], ck_c[used])


def test_autograd_function(setup):
    mech, m, o = setup
    f = synth.field(0, mech, 64)
    T0, p, Y0 = _dev(f)
    T0.requires_grad_(True)
    Y0.requires_grad_(True)
    lnA = torch.tensor(np.log([r["A"] for r in mech["reactions"]]), device=DEV, requires_grad=True)
    T, Y, q, st = df.chem_step(m, T0, p, Y0, lnA, f["dt"])
    loss = T.sum() + 1e-9 * q.sum()
    loss.backward()
    r = df.adjoint(m, T0.detach(), p, Y0.detach(), f["dt"], gT1=torch.ones_like(T),
                   gQ1=torch.full_like(T, 1e-9))
    assert torch.allclose(T0.grad, r["gT0"], rtol=1e-12, atol=0)
    assert torch.allclose(lnA.grad, r["g_lnA"], rtol=1e-12, atol=1e-300)
    # a finite-difference look at the adaptive map itself (its step sequence does
    # not change for a 1e-6 change of ln A on these cells)
    j = int(torch.argmax(lnA.grad.abs()))
    # (step 1e-4: sum(T) ~ 8e4 K carries ~1e-11 K of rounding, too much for 1e-6)
    vals = []
    for sgn in (1, -1):
        la = lnA.detach().clone()
        la[j] += sgn * 1e-4
        T2, Y2, q2, _ = df.chem_step(m, T0.detach(), p, Y0.detach(), la, f["dt"])
        vals.append((T2.sum() + 1e-9 * q2.sum()).item())
    fd = (vals[0] - vals[1]) / 2e-4
    assert abs(fd - lnA.grad[j].item()) <= 1e-3 * abs(fd) + 1e-9
    m.set_lnA(None)


@pytest.mark.parametrize("cfg", [1, 3])
def test_adjoint_every_component_against_oracle(setup, cfg):
    """Every component, not a projection: for single cells, each of the N + 1
    entries of (dL/dT0, dL/dY0) and each of the M entries of dL/d ln A against
    the oracle's complex-step derivative of the same replayed RODAS4 map along
    that unit direction.  Bound per entry: 1e-6 of itself plus 1e-9 of the
    largest entry of its vector (entries that vanish up to rounding)."""
    mech, m, o = setup
    N, M = m.n_species, m.n_reactions
    f = synth.field(cfg, mech, 64, seed=300 + cfg)
    rng = np.random.default_rng(301)
    for c in (0, 17, 40, 63):
        T, p, Y = (torch.tensor(np.ascontiguousarray(f[k][..., c:c + 1]), device=DEV) for k in ("T", "p", "Y"))
        gT, gY, gQ = rng.standard_normal(1), rng.standard_normal((N, 1)), rng.standard_normal(1) * 1e-9
        r = df.adjoint(m, T, p, Y, f["dt"], torch.tensor(gT, device=DEV), torch.tensor(gY, device=DEV),
                       torch.tensor(gQ, device=DEV))
        assert int(r["status"].abs().sum()) == 0
        hs = _steps(r, N, 0)
        y0 = np.concatenate([[f["T"][c]], f["Y"][:, c]])
        g_state = np.r_[r["gT0"].cpu().numpy(), r["gY0"].cpu().numpy()[:, 0]]
        g_lnA = r["g_lnA"].cpu().numpy()
        ref_state = np.array([o.ros_replay_dir(f["p"][c], y0, hs, wT=gT[0], wY=gY[:, 0], wQ=gQ[0],
                                               dy0=np.eye(N + 1)[i]) for i in range(N + 1)])
        ref_lnA = np.array([o.ros_replay_dir(f["p"][c], y0, hs, wT=gT[0], wY=gY[:, 0], wQ=gQ[0],
                                             dlnA=np.eye(M)[j]) for j in range(M)])
        for g, ref, name in ((g_state, ref_state, "state"), (g_lnA, ref_lnA, "lnA")):
            bound = 1e-6 * np.abs(ref) + 1e-9 * np.abs(ref).max()
            err = np.abs(g - ref)
            assert np.all(err <= bound), (cfg, c, name, int(np.argmax(err / bound)), float(np.max(err / bound)))
