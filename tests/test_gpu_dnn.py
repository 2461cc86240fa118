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
    d = np.abs(U[:, :9] - Uo[:, :9]) / scale
    # Same rounding points on both sides: the outputs differ only where an FP32
    # accumulation-order difference flips a BF16 rounding of a hidden
    # activation upstream (one BF16 ulp, 2^-8 relative, of one term of the
    # next layer's sums).  Bounds: the largest difference, and the share of
    # outputs touched by a flip at all (above the FP32 accumulation noise).
    # A flip in the last hidden layer moves an output by one BF16 ulp (2^-8 ..
    # 2^-7 relative) of one term W4_kj H3_j: a few 1e-3 of the scale at most.
    # Flips are rare per activation (FP32 accumulation noise of a K = 1600 sum,
    # ~1e-6 relative, and the GELU's ~3e-7, against a BF16 half-ulp of 2e-3), but
    # a row of the full network has 2800 activations: at most 40% of its rows
    # may be touched at all; the median output is exact to FP32 noise.
    touched = float(np.mean(d > 1e-5))
    print({"widths": widths, "rows": rows, "max": float(d.max()), "median": float(np.median(d)),
           "touched": touched})
    assert d.max() <= 4e-3, d.max()
    assert np.median(d) <= 1e-6
    assert touched <= (0.4 if widths[0] >= 1000 else 0.05)


@pytest.fixture(scope="module")
def data():
    mech = synth.h2_air_mechanism()
    m = df.Mechanism(mech)
    Ts, p, Ys = surrogate.trajectories(m, mech, 512, 4)
    return mech, m, surrogate.pairs(Ts, p, Ys)


# 512 rows and widths up to 64: the one-tile-per-CTA kernels; 1500 rows and
# widths 200 / 136 / 72: the persistent kernel's training epilogues (several
# row tiles per CTA, a ragged last row tile and a last 8-column chunk per layer)
@pytest.mark.parametrize("widths,n", [((64, 32, 16), 512), ((200, 136, 72), 1500)])
def test_train_step_gradients_match_oracle(data, widths, n):
    mech, m, (T0, P, Y0, T1, Y1) = data
    assert T0.shape[0] >= n
    dnn = df.Dnn(_opts(widths, batch=n), seed=3)
    dnn.fit_norm(T0, P, Y0, Y1)
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
    lo, go, _, cache = mlp.loss_and_grads(mlp.unpack(params0, widths), x, tgt, 9, emulate=True,
                                          return_cache=True)
    assert abs(loss - lo) <= 2e-3 * lo
    # Element by element, each weight gradient against the scale of its own
    # sum: dW_l[i, j] = sum_r dZ_l[r, i] H_{l-1}[r, j], S = sum_r |dZ_l| |H_{l-1}|.
    # The two sides agree up to FP32 accumulation order and the BF16 rounding
    # flips it causes upstream (each flip moves one term by 2^-8 of itself).
    worst = {}
    for l in (1, 2, 3, 4):
        dZ, H = np.abs(cache[f"dZ{l}"]), np.abs(cache[f"H{l - 1}"])
        SW = dZ.T @ H
        Sb = dZ.sum(axis=0)
        for name, S in ((f"W{l}", SW), (f"b{l}", Sb)):
            err = np.abs(g[name] - go[name])
            ok = err <= 2 ** -7 * S + 1e-9 * S.max()
            worst[name] = float((err / (S + 1e-300)).max())
            assert ok.all(), (name, worst[name], int((~ok).sum()))
            # and relative to the gradient itself where it is not a cancellation
            big = (np.abs(go[name]) >= 0.1 * S) & (S > 0)
            if big.any():
                rel = err[big] / np.abs(go[name][big])
                worst[name + "_rel"] = float(rel.max())
                assert np.median(rel) <= 1e-3, (name, float(np.median(rel)))
    print(worst)


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
    inert = mlp.inert_species(mech)
    To, Yo = mlp.post(f["T"][net], f["p"][net], f["Y"][:, net], U, 0.1, norm, 9, o.nasa, o.W, inert=inert)
    Yg = Y.cpu().numpy()[:, net]
    assert np.allclose(Yg.sum(axis=0), 1.0, rtol=1e-13)
    assert inert.sum() == 1 and np.array_equal(Yg[inert], f["Y"][inert][:, net])  # N2 untouched
    # same network, same rounding points: differences only where an FP32 / BF16
    # rounding decision flips between the two accumulation orders
    err = np.abs(Yg - Yo).max(axis=0) / (np.abs(Yo - f["Y"][:, net]).max() + 1e-300)
    assert np.median(err) <= 1e-4 and np.quantile(err, 0.99) <= 3e-3 and err.max() <= 3e-2
    for c in range(0, len(net), 97):
        cc = net[c]
        h0 = o.enthalpy_mass(f["T"][cc], f["Y"][:, cc])
        h1 = o.enthalpy_mass(T.cpu().numpy()[cc], Yg[:, c])
        assert abs(h1 - h0) <= 1e-9 * 1.5e3 * f["T"][cc]


def test_infer_full_size_sampled(data):
    """The inference pass at the size the bench times: 2^22 cells in the
    default 262144-row chunks through the 11-1600-800-400-9 network, 2% of
    them above the training T range.  Sampled network cells against the oracle
    pipeline (features, BF16-rounded MLP, post stage) and sampled fallback
    cells against a direct integration of the same cells (bitwise)."""
    mech, m, (T0, P, Y0, T1, Y1) = data
    dnn = df.Dnn(df.dnn_default_opts(), seed=13)
    dnn.fit_norm(T0, P, Y0, Y1)
    o = Mech(mech)
    n = 1 << 22
    f = synth.field(1, mech, n, seed=2024)
    f["T"] = np.clip(f["T"], T0.min().item() + 1, T0.max().item() - 1)
    rng = np.random.default_rng(5)
    out = np.sort(rng.choice(n, n // 50, replace=False))
    f["T"][out] = rng.uniform(T0.max().item() + 50.0, T0.max().item() + 300.0, out.size)
    T, p, Y = (torch.tensor(f[k], device=DEV) for k in ("T", "p", "Y"))
    nfb, used, status = dnn.infer(m, T, p, Y, f["dt"])
    used = used.cpu().numpy()
    # the moved cells and any other cell with a feature outside the training range
    fbl = np.nonzero(used)[0]
    assert nfb == fbl.size and np.all(used[out] == 1)
    assert int(status.abs().sum()) == 0
    Tg, Yg = T.cpu().numpy(), Y.cpu().numpy()
    # about 300 sampled fallback cells: a direct integration, bitwise
    fb = fbl[:: max(1, fbl.size // 300)]
    Ti, pi, Yi = (torch.tensor(np.ascontiguousarray(f[k][..., fb]), device=DEV) for k in ("T", "p", "Y"))
    df.integrate(m, Ti, pi, Yi, f["dt"])
    assert np.array_equal(Tg[fb], Ti.cpu().numpy()) and np.array_equal(Yg[:, fb], Yi.cpu().numpy())
    # sampled network cells, spread over every chunk
    net = np.arange(0, n, 9973)
    net = net[used[net] == 0]
    assert net.size > 300
    nm = dnn.norm()
    norm = {"mean_in": np.r_[nm["mean_in"], np.zeros(5)], "std_in": np.r_[nm["std_in"], np.ones(5)],
            "mean_out": np.r_[nm["mean_out"], np.zeros(7)], "std_out": np.r_[nm["std_out"], np.ones(7)]}
    _, x = mlp.features(f["T"][net], f["p"][net], f["Y"][:, net], 0.1, norm, 9)
    U, _ = mlp.forward(mlp.unpack(dnn.params(), (1600, 800, 400)), x.astype(np.float32), emulate=True)
    inert = mlp.inert_species(mech)
    To, Yo = mlp.post(f["T"][net], f["p"][net], f["Y"][:, net], U, 0.1, norm, 9, o.nasa, o.W, inert=inert)
    assert np.allclose(Yg[:, net].sum(axis=0), 1.0, rtol=1e-13)
    assert np.array_equal(Yg[inert][:, net], f["Y"][inert][:, net])
    err = np.abs(Yg[:, net] - Yo).max(axis=0) / (np.abs(Yo - f["Y"][:, net]).max() + 1e-300)
    print({"cells": n, "fallback": int(nfb), "sampled": len(net), "median": float(np.median(err)),
           "max": float(err.max())})
    assert np.median(err) <= 1e-4 and np.quantile(err, 0.99) <= 3e-3 and err.max() <= 3e-2


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
    To, Yo = mlp.post(Th[net], ph[net], Yh[:, net], U, 0.1, norm, 9, o.nasa, o.W,
                      inert=mlp.inert_species(mech))
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


def test_adam_steps_match_oracle(data):
    """Two training steps with lr > 0: the FP32 parameters and both moment
    estimates after each step against the oracle's Adam (Kingma & Ba,
    Algorithm 1, FP64) applied to the step's own gradient and the state the
    GPU held before the step."""
    mech, m, (T0, P, Y0, T1, Y1) = data
    widths = (64, 32, 16)
    dnn = df.Dnn(_opts(widths, batch=512), seed=4)
    dnn.fit_norm(T0, P, Y0, Y1)
    n, lr = 512, 3e-3
    theta = dnn.params().astype(np.float64)
    m1, m2, t = (a.astype(np.float64) if isinstance(a, np.ndarray) else a for a in dnn.adam_state())
    assert t == 0 and not m1.any() and not m2.any()
    for step in (1, 2):
        sl = slice((step - 1) * n, step * n)
        dnn.train_step(T0[sl].contiguous(), P[sl].contiguous(), Y0[:, sl].contiguous(), Y1[:, sl].contiguous(), lr)
        g = dnn.grads().astype(np.float64)
        th_o, m_o, v_o = mlp.adam_step(theta, m1, m2, g, step, lr)
        # FP32 roundings are relative to the two terms of each moment update,
        # not to the result (beta m and (1 - beta) g can cancel)
        sm = 0.9 * np.abs(m1) + 0.1 * np.abs(g)
        sv = 0.999 * m2 + 0.001 * g * g
        theta = dnn.params().astype(np.float64)
        a, b, t = dnn.adam_state()
        m1, m2 = a.astype(np.float64), b.astype(np.float64)
        assert t == step
        assert np.all(np.abs(m1 - m_o) <= 1e-6 * sm + 1e-30), np.max(np.abs(m1 - m_o) / (sm + 1e-30))
        assert np.all(np.abs(m2 - v_o) <= 1e-6 * sv + 1e-38), np.max(np.abs(m2 - v_o) / (sv + 1e-38))
        # FP32 parameter: one rounding of theta (half an ulp) plus the FP32
        # update's few roundings (relative 1e-6 of a step of size ~lr)
        tol = 2.0 ** -23 * np.abs(th_o) + 1e-6 * lr
        err = np.abs(theta - th_o)
        assert np.all(err <= tol), (step, float(np.max(err / tol)))
        assert np.max(np.abs(theta - th_o)) < 0.1 * lr


def test_gradient_halves_sum_to_the_union_gradient(data):
    """df_dnn_grad on two shards of a batch, each normalised by the whole batch,
    sums to the gradient of one pass over the union (FP32 summation order
    only: every row's output gradient is rounded to BF16 identically); then
    df_dnn_adam_step on the summed buffer gives the parameters of
    df_dnn_train_step on the union."""
    mech, m, (T0, P, Y0, T1, Y1) = data
    widths = (64, 32, 16)
    n = 512
    args = [a[..., :n].contiguous() for a in (T0, P, Y0, Y1)]
    ref = df.Dnn(_opts(widths, batch=512), seed=9)
    ref.fit_norm(T0, P, Y0, Y1)
    p0 = ref.params()
    lu = ref.grad(*args)
    g_union = ref.grad_tensor().clone()
    acc = torch.zeros_like(g_union)
    ls = 0.0
    for lo, hi in ((0, 200), (200, n)):
        ls += ref.grad(*[a[..., lo:hi].contiguous() for a in args], n_total=n)
        acc += ref.grad_tensor()
    assert abs(ls - lu) <= 1e-5 * lu
    scale = g_union.abs().max().item()
    assert torch.max(torch.abs(acc - g_union)).item() <= 1e-5 * scale
    # the split step on the summed gradient equals the fused step
    ref.grad_tensor().copy_(acc)
    ref.adam_step(1e-3)
    p_split = ref.params()
    fused = df.Dnn(_opts(widths, batch=512), seed=9)
    fused.fit_norm(T0, P, Y0, Y1)
    assert np.array_equal(fused.params(), p0)
    fused.train_step(*args, lr=1e-3)
    assert np.max(np.abs(p_split - fused.params())) <= 1e-6 * 1e-3 + 2 ** -22 * np.abs(p0).max()


def _element_imbalance(mech, Y0, Y1):
    """Largest relative change of the element mass per unit mass (moles of each
    element per kg), over cells: |sum_k a_ek (Y1_k - Y0_k) / W_k| /
    sum_k a_ek Y0_k / W_k."""
    names = [s["name"] for s in mech["species"]]
    elems = sorted({e for s in mech["species"] for e in s["composition"]})
    A = np.array([[s["composition"].get(e, 0) / s["W"] for s in mech["species"]] for e in elems])
    b0 = A @ Y0
    return np.max(np.abs(A @ (Y1 - Y0)) / np.maximum(b0, 1e-300), axis=0), names


@pytest.fixture(scope="module")
def trained():
    """The full 11-1600-800-400-9 network trained for 20 s on integrator pairs
    of the uneven-stiffness field (2^14 trajectories x 16 steps)."""
    mech = synth.h2_air_mechanism()
    m = df.Mechanism(mech)
    Ts, p, Ys = surrogate.trajectories(m, mech, 1 << 14, 16)
    T0, P0, Y0, T1, Y1 = surrogate.pairs(Ts, p, Ys)
    del Ts, Ys
    o = df.dnn_default_opts()
    dnn = df.Dnn(o, seed=22)
    dnn.fit_norm(T0, P0, Y0, Y1)
    surrogate.train(dnn, T0, P0, Y0, Y1, epochs=10_000, batch=4096, time_budget=20.0)
    return mech, m, dnn


def test_dnn_error_within_the_stated_per_species_bound(trained):
    """On 2^16 held-out trajectory states (no out-of-range cells): for every
    species the network's mean absolute error in Y(t + dt) against the FP64
    integrator is at most surrogate.ERROR_BOUND (10%) of the mean absolute
    change the integrator makes; the inert species is exact; the mean error in
    T is within the same fraction of the mean temperature change."""
    mech, m, dnn = trained
    Ts, p, Ys = surrogate.trajectories(m, mech, 1 << 12, 16, seed=4242)
    T = torch.cat(Ts[1:]).contiguous()
    Y = torch.cat(Ys[1:], dim=1).contiguous()
    P = p.repeat(len(Ts) - 1).contiguous()
    assert T.numel() >= 1 << 16
    ev = surrogate.evaluate(dnn, m, T, P, Y, mech_json=mech)
    print({k: (v.tolist() if hasattr(v, "tolist") else v) for k, v in ev.items() if k in
           ("mae_Y", "frozen_mae_Y", "max_Y", "mae_T", "frozen_mae_T", "n_fallback", "element_imbalance_dnn",
            "element_imbalance_integrator")})
    assert ev["n_network"] >= 0.95 * ev["n"]
    check = surrogate.within_bound(ev, surrogate.inert_mask(mech))
    assert check["ok"], check
