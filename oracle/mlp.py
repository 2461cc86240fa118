"""CPU oracle of the DNN chemistry integrator.  TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this module.  It shares no code with the CUDA path.

What it computes (numpy, FP64 unless a rounding point says otherwise):
  * the input encoding of Sec. 2.3: x = {T, p, F(Y_1..Y_N)} with the Box-Cox
    transform F(Y) = (max(Y, 0)^lambda - 1)/lambda, z-scored with the training
    statistics; the target is the change of F(Y) over dt, z-scored;
  * a fully connected network with three hidden layers (Sec. 2.3), exact-erf
    GELU, and its gradient for the mean-squared error;
  * stage 3 of DNNInferencer.inference (Sec. 3.2): Y' = F^{-1}(F(Y) + u),
    renormalised, and T' from h(T', Y') = h(T, Y) at fixed p (correctThermo);
    species that no reaction changes (net stoichiometric coefficient zero in
    every reaction, e.g. an inert collider) keep their input mass fraction and
    the renormalisation acts on the others (the paper is silent; this keeps
    dY_k/dt = 0 for those species exact, as the kinetics has it);
  * the optimiser the paper leaves open (Sec. 2.3 says only that the network
    is trained): Adam, Kingma & Ba 2015, Algorithm 1, with bias-corrected
    first and second moments, in FP64 on the FP32 master weights.

Rounding points (``emulate=True``) follow the GPU path: features rounded to
FP32 then to BF16, weights BF16, products accumulated in FP64 here (FP32 on
the GPU), bias + GELU in FP32, activations rounded to BF16 (round to nearest
even); in the backward pass dU, dZ = (dH * gelu'(Z)) are rounded to BF16.
``emulate=False`` is the exact FP64 network, pinned by finite differences.

Parity status: pinned (tests/test_oracle_mlp.py: finite differences of the
exact network; BF16 rounding against a library conversion; the Box-Cox
features against hand-computed values; Adam against a hand-worked two-step
example and its closed-form first step; the post stage against its fixed
points and the inert-species rule).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

DNN_IN = 16
DNN_OUT = 16


def bf16(x) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even); float32 result."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    nan = np.isnan(a)
    if nan.any():
        out = out.copy()
        out[nan] = np.nan
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def layout(widths):
    """(name, shape) of the parameters in the GPU's flat order."""
    w1, w2, w3 = widths
    return [("W1", (w1, DNN_IN)), ("b1", (w1,)), ("W2", (w2, w1)), ("b2", (w2,)),
            ("W3", (w3, w2)), ("b3", (w3,)), ("W4", (DNN_OUT, w3)), ("b4", (DNN_OUT,))]


def unpack(flat, widths):
    out, o = {}, 0
    for name, shp in layout(widths):
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(p, widths):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in layout(widths)])


def features(T, p, Y, lam, norm, N):
    """Features [n, 16]: T, p, F(Y_k) (F in FP64), rounded to FP32 and z-scored in
    FP32 with the FP32 statistics (the GPU's rounding points before BF16)."""
    n = T.shape[0]
    f = np.zeros((n, DNN_IN))
    f[:, 0] = T
    f[:, 1] = p
    f[:, 2:2 + N] = ((np.maximum(Y, 0.0).T) ** lam - 1.0) / lam
    f32 = f.astype(np.float32)
    x = np.zeros_like(f32)
    mean = np.asarray(norm["mean_in"], np.float32)[:2 + N]
    std = np.asarray(norm["std_in"], np.float32)[:2 + N]
    x[:, :2 + N] = (f32[:, :2 + N] - mean) / std
    return f, x


def forward(params, X, emulate=True):
    """Network output U [n, 16] and the cache for backward.  X: [n, 16]."""
    P = params
    H = bf16(X).astype(np.float64) if emulate else np.asarray(X, np.float64)
    cache = {"H0": H}
    for l in (1, 2, 3):
        W = bf16(P[f"W{l}"]).astype(np.float64) if emulate else P[f"W{l}"]
        Z = H @ W.T + (P[f"b{l}"].astype(np.float32).astype(np.float64) if emulate else P[f"b{l}"])
        if emulate:
            Z = Z.astype(np.float32).astype(np.float64)
        G = gelu(Z)
        H = bf16(G).astype(np.float64) if emulate else G
        cache[f"Z{l}"] = Z
        cache[f"H{l}"] = H
    W4 = bf16(P["W4"]).astype(np.float64) if emulate else P["W4"]
    U = H @ W4.T + P["b4"]
    if emulate:
        U = U.astype(np.float32).astype(np.float64)
    return U, cache


def loss_and_grads(params, X, tgt, N, emulate=True, return_cache=False):
    """Mean squared error over the first N outputs and its parameter gradients.
    return_cache: also return the forward cache and the backward products
    dZ_l (and dU), for scale estimates in tests."""
    P = params
    n = X.shape[0]
    U, c = forward(P, X, emulate)
    d = U[:, :N] - tgt[:, :N]
    loss = float(np.sum(d * d) / (n * N))
    dU = np.zeros_like(U)
    dU[:, :N] = 2.0 * d / (n * N)
    if emulate:
        dU = bf16(dU).astype(np.float64)
    g = {}
    g["W4"] = dU.T @ c["H3"]
    g["b4"] = dU.sum(axis=0)
    W = {l: (bf16(P[f"W{l}"]).astype(np.float64) if emulate else P[f"W{l}"]) for l in (1, 2, 3, 4)}
    dH = dU @ W[4]
    c["dZ4"] = dU
    for l in (3, 2, 1):
        dZ = dH * gelu_grad(c[f"Z{l}"])
        if emulate:
            dZ = bf16(dZ).astype(np.float64)
        c[f"dZ{l}"] = dZ
        g[f"W{l}"] = dZ.T @ c[f"H{l - 1}"]
        g[f"b{l}"] = dZ.sum(axis=0)
        dH = dZ @ W[l]
    if return_cache:
        return loss, g, U, c
    return loss, g, U


def inert_species(mech: dict) -> np.ndarray:
    """Species whose net stoichiometric coefficient is zero in every reaction
    of the mechanism (Sec. 2.3 eq. (sourceeq): their production rate is then
    identically zero).  Boolean [N] in the mechanism's species order."""
    names = [sp["name"] for sp in mech["species"]]
    net = np.zeros(len(names))
    seen = np.zeros(len(names), bool)
    for r in mech["reactions"]:
        nu = np.zeros(len(names))
        for side, sgn in (("reactants", -1.0), ("products", 1.0)):
            for name, c in r[side].items():
                nu[names.index(name)] += sgn * c
        seen |= nu != 0.0
    return ~seen


def adam_step(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1), FP64:
    m <- beta1 m + (1 - beta1) g;  v <- beta2 v + (1 - beta2) g^2;
    m_hat = m / (1 - beta1^t);  v_hat = v / (1 - beta2^t);
    theta <- theta - lr m_hat / (sqrt(v_hat) + eps).   t counts from 1.
    Returns (theta, m, v)."""
    theta, m, v, g = (np.asarray(a, np.float64) for a in (theta, m, v, g))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def post(T, p, Y, U, lam, norm, N, nasa, W, inert=None):
    """Stage 3 of the inference (FP64): Y' = F^{-1}(F(Y) + u) renormalised, and T'
    with h(T', Y') = h(T, Y).  nasa [N, 7], W [N] (g/mol).  inert [N] (bool,
    optional): species kept at their input mass fraction; the others are
    scaled so that the mass fractions sum to one."""
    u = U[:, :N] * norm["std_out"][:N] + norm["mean_out"][:N]
    z = np.maximum(Y.T, 0.0) ** lam + lam * u
    Yn = np.where(z > 0, np.maximum(z, 0.0) ** (1.0 / lam), 0.0)
    if inert is None or not np.any(inert):
        Yn = Yn / Yn.sum(axis=1, keepdims=True)
    else:
        inert = np.asarray(inert, bool)
        Yn[:, inert] = Y.T[:, inert]
        rest = 1.0 - Yn[:, inert].sum(axis=1, keepdims=True)
        Yn[:, ~inert] = Yn[:, ~inert] * (rest / Yn[:, ~inert].sum(axis=1, keepdims=True))

    def h_mass(Tk, Yk):  # h / R per unit mass, sum_k Y_k/W_k * H_k/R
        a = nasa
        hRT = (a[:, 0] + Tk[:, None] * (a[:, 1] / 2 + Tk[:, None] * (a[:, 2] / 3 + Tk[:, None] *
               (a[:, 3] / 4 + Tk[:, None] * a[:, 4] / 5))) + a[:, 5] / Tk[:, None])
        return np.sum(Yk / W * hRT * Tk[:, None], axis=1)

    def cp_mass(Tk, Yk):
        a = nasa
        cpR = a[:, 0] + Tk[:, None] * (a[:, 1] + Tk[:, None] * (a[:, 2] + Tk[:, None] *
                                                               (a[:, 3] + Tk[:, None] * a[:, 4])))
        return np.sum(Yk / W * cpR, axis=1)

    h0 = h_mass(T, Y.T)
    Tn = T.copy()
    for _ in range(30):
        dT = (h_mass(Tn, Yn) - h0) / cp_mass(Tn, Yn)
        Tn = Tn - dT
        if np.max(np.abs(dT) / Tn) < 1e-14:
            break
    return Tn, Yn.T
