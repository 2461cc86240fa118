"""Pins of the CPU MLP oracle: finite differences of the exact network, the
BF16 rounding against a library conversion, the inverse transform and the
enthalpy Newton against their definitions' fixed points."""
import numpy as np
import pytest

from oracle import mlp
from oracle.oracle import Mech
from paper_2210_07094_gb300 import synth


def _params(widths, seed=0):
    rng = np.random.default_rng(seed)
    flat = []
    for name, shp in mlp.layout(widths):
        flat.append(rng.standard_normal(shp).ravel() * (0.5 if name.startswith("W") else 0.1))
    return mlp.unpack(np.concatenate(flat), widths)


def test_bf16_rounding_matches_library():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(100000).astype(np.float32) * 10 ** rng.uniform(-30, 30, 100000),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.0078125, 3.0e38], np.float32)]).astype(np.float32)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_exact_gradients_vs_finite_differences():
    """Tiny net (3 inputs -> 8 -> 8 -> 8 -> 2 outputs), exact FP64 mode."""
    widths = (8, 8, 8)
    P = _params(widths)
    P["W1"][:, 3:] = 0.0  # 3 real inputs
    P["W4"][2:, :] = 0.0
    P["b4"][2:] = 0.0
    rng = np.random.default_rng(2)
    X = np.zeros((5, mlp.DNN_IN))
    X[:, :3] = rng.standard_normal((5, 3))
    tgt = np.zeros((5, mlp.DNN_OUT))
    tgt[:, :2] = rng.standard_normal((5, 2))
    loss, g, _ = mlp.loss_and_grads(P, X, tgt, 2, emulate=False)
    flat = mlp.pack(P, widths)
    gflat = mlp.pack(g, widths)
    idx = rng.choice(flat.size, 60, replace=False)
    for i in idx:
        e = 1e-6
        fp, fm = flat.copy(), flat.copy()
        fp[i] += e
        fm[i] -= e
        lp = mlp.loss_and_grads(mlp.unpack(fp, widths), X, tgt, 2, emulate=False)[0]
        lm = mlp.loss_and_grads(mlp.unpack(fm, widths), X, tgt, 2, emulate=False)[0]
        fd = (lp - lm) / (2 * e)
        assert abs(gflat[i] - fd) <= 1e-7 * max(1.0, abs(fd)), (i, gflat[i], fd)


def test_emulated_network_is_close_to_exact():
    widths = (64, 32, 16)
    P = _params(widths, 3)
    X = np.random.default_rng(4).standard_normal((50, mlp.DNN_IN))
    Ue, _ = mlp.forward(P, X, emulate=True)
    Ux, _ = mlp.forward(P, X, emulate=False)
    assert np.max(np.abs(Ue - Ux)) <= 0.05 * np.max(np.abs(Ux))


def test_post_inverts_the_transform_and_keeps_enthalpy():
    """u = 0 returns the input state; a nonzero u keeps h(T, Y) fixed."""
    mech = synth.h2_air_mechanism()
    o = Mech(mech)
    f = synth.field(1, mech, 20)
    N = 9
    norm = {"mean_out": np.zeros(16), "std_out": np.ones(16)}
    U0 = np.zeros((20, 16))
    T1, Y1 = mlp.post(f["T"], f["p"], f["Y"], U0, 0.1, norm, N, o.nasa, o.W)
    assert np.allclose(Y1, f["Y"] / f["Y"].sum(axis=0), rtol=1e-12, atol=1e-300)
    assert np.allclose(T1, f["T"], rtol=1e-12)
    U = np.zeros((20, 16))
    U[:, :N] = np.random.default_rng(5).standard_normal((20, N)) * 0.01
    T2, Y2 = mlp.post(f["T"], f["p"], f["Y"], U, 0.1, norm, N, o.nasa, o.W)
    for c in range(20):
        assert abs(o.enthalpy_mass(T2[c], Y2[:, c]) - o.enthalpy_mass(f["T"][c], f["Y"][:, c])) <= \
            1e-9 * 1.5e3 * f["T"][c]
    assert np.allclose(Y2.sum(axis=0), 1.0, rtol=1e-14)


def test_box_cox_features_hand_values():
    """F(Y) = (max(Y, 0)^lambda - 1) / lambda at lambda = 0.1 (Sec. 2.3, Box-Cox):
    F(1) = 0, F(0) = -1/lambda, F(1e-6) = (10^-0.6 - 1)/0.1, F(0.01) = (10^-0.2 - 1)/0.1,
    a negative mass fraction clipped to F(0); then the z-score in FP32."""
    N = 5
    Y = np.array([[1.0], [0.0], [1e-6], [0.01], [-1e-3]])
    T = np.array([1500.0])
    p = np.array([101325.0])
    norm = {"mean_in": np.r_[1200.0, 101325.0, -5.0, -5.0, -5.0, -5.0, -5.0, np.zeros(9)],
            "std_in": np.r_[300.0, 1.0, 2.5, 2.5, 2.5, 2.5, 2.5, np.ones(9)]}
    f, x = mlp.features(T, p, Y, 0.1, norm, N)
    expect_F = [0.0, -10.0, -7.4881135684904199, -3.6904265551980675, -10.0]
    assert f[0, 0] == 1500.0 and f[0, 1] == 101325.0
    assert np.allclose(f[0, 2:2 + N], expect_F, rtol=1e-14, atol=1e-14)
    # z-score in FP32: (1500 - 1200)/300 = 1, (101325 - 101325)/1 = 0, (F + 5)/2.5
    assert x.dtype == np.float32
    assert x[0, 0] == np.float32(1.0) and x[0, 1] == np.float32(0.0)
    zs = [(np.float32(v) - np.float32(-5.0)) / np.float32(2.5) for v in expect_F]
    assert np.allclose(x[0, 2:2 + N], zs, rtol=2e-7, atol=2e-7)
    assert np.all(x[0, 2 + N:] == 0.0)


def test_adam_hand_worked_two_steps():
    """theta0 = 1, gradients 0.5 then -0.25, lr 0.1, beta 0.9 / 0.999, eps 1e-8
    (Kingma & Ba 2015, Algorithm 1), worked by hand in exact fractions:
    step 1: m = 1/20, v = 1/4000, m_hat = 1/2, v_hat = 1/4,
            theta = 1 - 0.1 * 0.5 / (0.5 + 1e-8) = 0.90000000199999996...
    step 2: m = 1/50, v = 1249/4000000, m_hat = 2/19, v_hat = 1249/7996,
            sqrt(v_hat) = 0.39522538070166418..., theta = 0.87336629870784616..."""
    th, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    th, m, v = mlp.adam_step(th, m, v, np.array([0.5]), 1, 0.1)
    # FP64 rounding of the decimal constants only: a few ulp
    assert abs(m[0] - 0.05) <= 4e-15 * 0.05 and abs(v[0] - 0.00025) <= 4e-15 * 0.00025
    assert abs(th[0] - 0.90000000199999996) <= 1e-15
    th, m, v = mlp.adam_step(th, m, v, np.array([-0.25]), 2, 0.1)
    assert abs(m[0] - 0.02) <= 4e-15 * 0.02 and abs(v[0] - 0.00031225) <= 4e-15 * 0.00031225
    assert abs(th[0] - 0.87336629870784616) <= 1e-15


def test_adam_closed_forms():
    """With the bias corrections, the first step moves every parameter by
    lr g/(|g| + eps) whatever beta1, beta2; a constant gradient keeps m_hat = g
    and v_hat = g^2 at every step, so every step moves by the same amount."""
    rng = np.random.default_rng(7)
    g = rng.standard_normal(1000) * 10 ** rng.uniform(-6, 2, 1000)
    th0 = rng.standard_normal(1000)
    for b1, b2 in ((0.9, 0.999), (0.5, 0.9)):
        th, m, v = mlp.adam_step(th0, np.zeros(1000), np.zeros(1000), g, 1, 1e-3, b1, b2)
        assert np.allclose(th, th0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    th, m, v = th0.copy(), np.zeros(1000), np.zeros(1000)
    for t in range(1, 51):
        th_prev = th
        th, m, v = mlp.adam_step(th, m, v, g, t, 1e-3)
        assert np.allclose(th_prev - th, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-18)


def test_inert_species_keep_their_mass_fraction():
    """N2 takes part in no reaction of the 9-species mechanism (a collider only),
    so its mass fraction must not change; the renormalisation acts on the rest
    and the mass fractions still sum to one."""
    mech = synth.h2_air_mechanism()
    inert = mlp.inert_species(mech)
    names = [s["name"] for s in mech["species"]]
    assert [names[k] for k in np.where(inert)[0]] == ["N2"]
    o = Mech(mech)
    f = synth.field(1, mech, 20)
    U = np.zeros((20, 16))
    U[:, :9] = np.random.default_rng(6).standard_normal((20, 9)) * 0.01
    norm = {"mean_out": np.zeros(16), "std_out": np.ones(16)}
    T2, Y2 = mlp.post(f["T"], f["p"], f["Y"], U, 0.1, norm, 9, o.nasa, o.W, inert=inert)
    assert np.array_equal(Y2[inert], f["Y"][inert])
    assert np.allclose(Y2.sum(axis=0), 1.0, rtol=1e-14)
    for c in range(20):
        assert abs(o.enthalpy_mass(T2[c], Y2[:, c]) - o.enthalpy_mass(f["T"][c], f["Y"][:, c])) <= \
            1e-9 * 1.5e3 * f["T"][c]
