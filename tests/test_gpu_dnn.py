"""DNN integrator on the GPU: layers against the CPU MLP oracle (same BF16
rounding points), gradients of one training step, the inference pipeline
(post-processing, enthalpy, fallback) and a short training run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2210_07094_gb300 as df  # noqa: E402
from oracle import mlp  # noqa: E402
from oracle.oracle import Mech  # noqa: E402
from paper_2210_07094_gb300 import surrogate, synth  # noqa: E402

DEV = "cuda:0"


def _opts(widths, batch=1024):
    o = df.dnn_default_opts()
    o.width[0], o.width[1], o.width[2] = widths
    o.batch = batch
    o.infer_chunk = 4096
    return o


# 1000 rows: one-tile-per-CTA kernels; 5000 rows (ragged last row block): the
# persistent kernels with the TMA-store epilogue
@pytest.mark.parametrize("widths,rows", [((32, 16, 8), 1000), ((1600, 800, 400), 1000),
                                         ((1600, 800, 400), 5000), ((200, 136, 72), 5000)])
def test_forward_matches_oracle(widths, rows):
    o = _opts(widths)
    o.infer_chunk = 8192
    dnn = df.Dnn(o, seed=5)
    P = mlp.unpack(dnn.params(), widths)
    rng = np.random.default_rng(0)
    Xf = np.zeros((rows, 16), np.float32)
    Xf[:, :11] = rng.standard_normal((rows, 11))
    X = torch.tensor(Xf, device=DEV).to(torch.bfloat16)
    U = dnn.forward_raw(X).cpu().numpy()
    Uo, _ = mlp.forward(P, X.float().cpu().numpy(), emulate=True)
    scale = np.abs(Uo[:, :9]).max()
    d = np.abs(U[:, :9] - Uo[:, :9])
    assert d.max() <= 1e-2 * scale, (d.max(), scale)
    assert d.mean() <= 1e-3 * scale


@pytest.fixture(scope="module")
def data():
    mech = synth.h2_air_mechanism()
    m = df.Mechanism(mech)
    Ts, p, Ys = surrogate.trajectories(m, mech, 512, 4)
    return mech, m, surrogate.pairs(Ts, p, Ys)


def test_train_step_gradients_match_oracle(data):
    mech, m, (T0, P, Y0, T1, Y1) = data
    widths = (64, 32, 16)
    dnn = df.Dnn(_opts(widths, batch=512), seed=3)
    dnn.fit_norm(T0, P, Y0, Y1)
    n = 512
    params0 = dnn.params()
    loss = dnn.train_step(T0[:n].contiguous(), P[:n].contiguous(), Y0[:, :n].contiguous(),
                          Y1[:, :n].contiguous(), lr=0.0)
    g = mlp.unpack(dnn.grads(), widths)
    assert np.array_equal(dnn.params(), params0)  # lr = 0
    nm = dnn.norm()
    norm = {"mean_in": np.r_[nm["mean_in"], np.zeros(5)], "std_in": np.r_[nm["std_in"], np.ones(5)],
            "mean_out": np.r_[nm["mean_out"], np.zeros(7)], "std_out": np.r_[nm["std_out"], np.ones(7)]}
    Tn, pn, Yn0, Yn1 = (a.cpu().numpy() for a in (T0[:n], P[:n], Y0[:, :n], Y1[:, :n]))
    f, x = mlp.features(Tn, pn, Yn0, 0.1, norm, 9)
    x = x.astype(np.float32)
    du = ((np.maximum(Yn1.T, 0) ** 0.1) - (np.maximum(Yn0.T, 0) ** 0.1)) / 0.1
    tgt = np.zeros((n, 16))
    tgt[:, :9] = (du - norm["mean_out"][:9]) / norm["std_out"][:9]
    lo, go, _ = mlp.loss_and_grads(mlp.unpack(params0, widths), x, tgt, 9, emulate=True)
    assert abs(loss - lo) <= 2e-3 * lo
    for name, _ in mlp.layout(widths):
        a, b = g[name], go[name]
        assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b) + 1e-12, name


# small widths, and the full 1600-800-400 network (its layers take the
# shared-memory-capped GEMM shapes while fallback blocks share the SMs)
@pytest.mark.parametrize("widths", [(32, 16, 8), (1600, 800, 400)])
def test_infer_pipeline_and_fallback(data, widths):
    mech, m, (T0, P, Y0, T1, Y1) = data
    dnn = df.Dnn(_opts(widths), seed=7)
    dnn.fit_norm(T0, P, Y0, Y1)
    o = Mech(mech)
    f = synth.field(1, mech, 3000, seed=99)
    f["T"] = np.clip(f["T"], T0.min().item() + 1, T0.max().item() - 1)
    out = np.array([5, 17, 400, 2999])
    f["T"][out] = 2900.0  # above the training range
    T, p, Y = (torch.tensor(f[k], device=DEV) for k in ("T", "p", "Y"))
    nfb, used, status = dnn.infer(m, T, p, Y, f["dt"])
    used = used.cpu().numpy()
    assert nfb >= len(out) and np.all(used[out] == 1)
    assert int(status.abs().sum()) == 0
    # fallback cells equal a direct integration of the same cells
    Ti, pi, Yi = (torch.tensor(np.ascontiguousarray(f[k][..., out]), device=DEV) for k in ("T", "p", "Y"))
    df.integrate(m, Ti, pi, Yi, f["dt"])
    assert np.array_equal(T.cpu().numpy()[out], Ti.cpu().numpy())
    # network cells: the oracle pipeline with the same network
    net = np.where(used == 0)[0]
    nm = dnn.norm()
    norm = {"mean_in": np.r_[nm["mean_in"], np.zeros(5)], "std_in": np.r_[nm["std_in"], np.ones(5)],
            "mean_out": np.r_[nm["mean_out"], np.zeros(7)], "std_out": np.r_[nm["std_out"], np.ones(7)]}
    _, x = mlp.features(f["T"][net], f["p"][net], f["Y"][:, net], 0.1, norm, 9)
    U, _ = mlp.forward(mlp.unpack(dnn.params(), widths), x.astype(np.float32), emulate=True)
    To, Yo = mlp.post(f["T"][net], f["p"][net], f["Y"][:, net], U, 0.1, norm, 9, o.nasa, o.W)
    Yg = Y.cpu().numpy()[:, net]
    assert np.allclose(Yg.sum(axis=0), 1.0, rtol=1e-13)
    # same network, same rounding points: differences only where an FP32 / BF16
    # rounding decision flips between the two accumulation orders
    err = np.abs(Yg - Yo).max(axis=0) / (np.abs(Yo - f["Y"][:, net]).max() + 1e-300)
    assert np.median(err) <= 1e-4 and np.quantile(err, 0.99) <= 3e-3 and err.max() <= 3e-2
    for c in range(0, len(net), 97):
        cc = net[c]
        h0 = o.enthalpy_mass(f["T"][cc], f["Y"][:, cc])
        h1 = o.enthalpy_mass(T.cpu().numpy()[cc], Yg[:, c])
        assert abs(h1 - h0) <= 1e-9 * 1.5e3 * f["T"][cc]


def test_post_resolves_small_changes(data):
    """Stage 3 on changes far below FP32 resolution of Y itself: with the output
    layer's weights zeroed the network returns its bias, so every cell gets the
    same small u (relative changes 1e-7 .. 1e-5 of Y).  Y' and T' must agree with
    the FP64 oracle post stage to a small fraction of the change."""
    mech, m, (T0, P, Y0, T1, Y1) = data
    widths = (32, 16, 8)
    dnn = df.Dnn(_opts(widths), seed=5)
    dnn.fit_norm(T0, P, Y0, Y1)
    dnn.set_norm(mean_out=np.zeros(9), std_out=np.ones(9))  # u = U: no de-normalisation rounding
    nm = dnn.norm()
    w = mlp.unpack(dnn.params(), widths)
    w["W4"][:] = 0.0
    w["b4"][:] = 0.0
    w["b4"][:9] = [1e-7 * (1 if k % 2 else -1) * (1 + 0.1 * k) for k in range(9)]
    dnn.set_params(mlp.pack(w, widths))
    o = Mech(mech)
    sel = np.arange(0, T0.numel(), 7)
    T, p, Y = T0[sel].clone(), P[sel].clone(), Y0[:, sel].clone().contiguous()
    Th, ph, Yh = T.cpu().numpy(), p.cpu().numpy(), Y.cpu().numpy()
    nfb, used, status = dnn.infer(m, T, p, Y, 1e-6)
    net = np.where(used.cpu().numpy() == 0)[0]
    assert len(net) > 0.9 * len(sel)
    U = np.tile(w["b4"].astype(np.float32), (len(net), 1)).astype(np.float64)
    norm = {"mean_out": np.r_[nm["mean_out"], np.zeros(7)], "std_out": np.r_[nm["std_out"], np.ones(7)]}
    To, Yo = mlp.post(Th[net], ph[net], Yh[:, net], U, 0.1, norm, 9, o.nasa, o.W)
    Yg, Tg = Y.cpu().numpy()[:, net], T.cpu().numpy()[net]
    dY = np.abs(Yo - Yh[:, net])
    assert dY.max() > 0
    assert np.all(np.abs(Yg - Yo) <= 1e-4 * dY + 1e-22), np.max(np.abs(Yg - Yo) / (dY + 1e-30))
    assert np.all(np.abs(Tg - To) <= 1e-3 * np.abs(To - Th[net]) + 1e-10 * Th[net])


def test_save_load_roundtrip(tmp_path):
    dnn = df.Dnn(_opts((32, 16, 8)), seed=11)
    path = str(tmp_path / "net.bin")
    dnn.save(path)
    d2 = df.Dnn.load(path)
    X = torch.randn(300, 16, device=DEV).to(torch.bfloat16)
    assert torch.equal(dnn.forward_raw(X), d2.forward_raw(X))


def test_short_training_learns_the_map(data):
    """A few hundred Adam steps: the loss falls, and on held-out trajectory states
    the network explains most of the variance of the change of F(Y) that the
    integrator computes (coefficient of determination over the reacting species)."""
    mech, m, (T0, P, Y0, T1, Y1) = data
    dnn = df.Dnn(_opts((256, 128, 64), batch=256), seed=1)
    dnn.fit_norm(T0, P, Y0, Y1)
    losses = surrogate.train(dnn, T0, P, Y0, Y1, epochs=40, batch=256, lr0=3e-3, lr1=1e-4)
    assert losses[-1][1] < 0.2 * losses[0][1]
    Ts, p, Ys = surrogate.trajectories(m, mech, 256, 2, seed=777)
    ev = surrogate.evaluate(dnn, m, Ts[1], p, Ys[1])
    assert ev["n_network"] > 0
    reacting = ev["var_dF"] > 0
    assert np.mean(ev["r2_dF"][reacting]) > 0.5, ev["r2_dF"]
