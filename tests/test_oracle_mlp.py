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
