"""Training data, training loop and evaluation of the DNN chemistry integrator.

The network learns the map the FP64 integrator computes (Sec. 2.3: the output
is the change of the Box-Cox-transformed input over one step dt, and the DNN
"can be regarded as an ODE integrator").  Training pairs are states along
integrator trajectories started from the uneven-stiffness field (bimodal T,
p 1-10 atm): each trajectory is advanced dt at a time by df_chem_integrate and
every (state, next state) pair is kept.  All arithmetic runs in the library's
kernels; this module only orchestrates calls.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import Dnn, Mechanism, dnn_default_opts, integrate, synth

# Acceptance bound of the learned integrator against the FP64 integrator on
# held-out states (the paper gives none; Sec. 4 compares DNN and CVODE results
# by eye): for every species, the mean absolute error of Y(t + dt) is at most
# this fraction of the mean absolute change the integrator makes over dt, the
# same for T; species that no reaction changes are exact.
ERROR_BOUND = 0.10


def inert_mask(mech_json: dict) -> np.ndarray:
    """Species whose net stoichiometric coefficient is zero in every reaction
    (their mass fraction cannot change)."""
    names = [sp["name"] for sp in mech_json["species"]]
    moves = np.zeros(len(names), bool)
    for r in mech_json["reactions"]:
        net = dict.fromkeys(names, 0)
        for name, c in r["reactants"].items():
            net[name] -= c
        for name, c in r["products"].items():
            net[name] += c
        for k, name in enumerate(names):
            moves[k] |= net[name] != 0
    return ~moves


def element_matrix(mech_json: dict) -> np.ndarray:
    """[elements, species]: atoms of each element per unit mass of each
    species, a_ek / W_k (mol/g)."""
    elems = sorted({e for sp in mech_json["species"] for e in sp["composition"]})
    return np.array([[sp["composition"].get(e, 0) / sp["W"] for sp in mech_json["species"]] for e in elems])


def within_bound(ev: dict, inert, bound: float = ERROR_BOUND) -> dict:
    """Check an evaluate() result against the acceptance bound; returns the
    per-species ratios and ok."""
    inert = np.asarray(inert, bool)
    ratio = ev["mae_Y"] / np.maximum(ev["frozen_mae_Y"], 1e-300)
    ok_species = np.where(inert, ev["max_Y"] == 0.0, ratio <= bound)
    ratio_T = ev["mae_T"] / max(ev["frozen_mae_T"], 1e-300)
    return {"ok": bool(ok_species.all() and ratio_T <= bound), "bound": bound,
            "mae_ratio_per_species": [float(x) for x in ratio], "inert_exact": bool(np.all(ev["max_Y"][inert] == 0)),
            "mae_ratio_T": float(ratio_T), "species_ok": [bool(x) for x in ok_species]}


def trajectories(mech: Mechanism, mech_json: dict, n_init: int, n_steps: int, dt: float = 1e-6,
                 seed: int = synth.TRAIN_SEED, device="cuda"):
    """States along integrator trajectories: returns device tensors T, p, Y of
    n_init * (n_steps + 1) states, trajectory-major in time (block s holds step s)."""
    import torch
    f = synth.field(1, mech_json, n_init, seed=seed)
    T = torch.tensor(f["T"], device=device)
    p = torch.tensor(f["p"], device=device)
    Y = torch.tensor(f["Y"], device=device)
    Ts, Ys = [T.clone()], [Y.clone()]
    for _ in range(n_steps):
        st, _ = integrate(mech, T, p, Y, dt)
        if int((st != 0).sum()) != 0:
            raise RuntimeError("integrator failed while generating training data")
        Ts.append(T.clone())
        Ys.append(Y.clone())
    return Ts, p, Ys


def pairs(Ts, p, Ys):
    """(state, next state) pairs from trajectory blocks: SoA device tensors."""
    import torch
    T0 = torch.cat(Ts[:-1])
    T1 = torch.cat(Ts[1:])
    P = p.repeat(len(Ts) - 1)
    Y0 = torch.cat(Ys[:-1], dim=1).contiguous()
    Y1 = torch.cat(Ys[1:], dim=1).contiguous()
    return T0, P, Y0, T1, Y1


def train(dnn: Dnn, T, p, Y, Yn, epochs: float, batch: int, lr0=1e-3, lr1=1e-5, seed=0, time_budget=None,
          log=None):
    """Adam with a cosine learning-rate schedule over shuffled mini-batches.
    Each epoch the pairs are permuted once into batch-major blocks, so every
    step hands the library contiguous views (no per-step gathers).  With a
    time budget the schedule spans the steps that fit in it: the step rate is
    measured over the first 200 steps and the cosine's length set from it, so
    the learning rate has decayed to lr1 when the budget ends.  The rate is
    taken over steps 200-400, after the one-time set-up of the first steps
    (the graph capture of the step)."""
    import torch
    n = T.numel()
    batch = min(batch, n)
    steps_per_epoch = max(1, n // batch)
    total = max(1, int(epochs * steps_per_epoch))
    probe0, probe = (200, 400) if time_budget is not None else (-1, -1)
    t_probe0 = None
    g = torch.Generator(device=T.device).manual_seed(seed)
    losses = []
    t0 = time.time()
    N = Y.shape[0]
    m = steps_per_epoch * batch
    for s in range(total):
        k = s % steps_per_epoch
        if k == 0:
            perm = torch.randperm(n, device=T.device, generator=g)[:m]
            Ts = T[perm].view(steps_per_epoch, batch)
            Ps = p[perm].view(steps_per_epoch, batch)
            Ys = Y[:, perm].view(N, steps_per_epoch, batch).permute(1, 0, 2).contiguous()
            Yns = Yn[:, perm].view(N, steps_per_epoch, batch).permute(1, 0, 2).contiguous()
        if s == probe0:
            torch.cuda.synchronize()
            t_probe0 = time.time()
        if s == probe:  # steps that fit in the budget at the measured rate
            torch.cuda.synchronize()
            now = time.time()
            rate = (probe - probe0) / max(now - t_probe0, 1e-9)
            total = min(total, max(s + 1, s + int(rate * (time_budget - (now - t0)))))
        lr = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * min(s / total, 1.0)))
        want = (s % 50 == 0) or s == total - 1
        loss = dnn.train_step(Ts[k], Ps[k], Ys[k], Yns[k], lr, want_loss=want)
        if want:
            losses.append((s, loss))
            if log:
                log(f"step {s}/{total} lr {lr:.2e} loss {loss:.4e}")
        if s + 1 >= total or (time_budget is not None and time.time() - t0 > 1.1 * time_budget):
            break
    return losses


def evaluate(dnn: Dnn, mech: Mechanism, T, p, Y, dt=1e-6, mech_json: dict | None = None):
    """Per-species error of the network against the integrator on the same states
    (in-range cells only), and the error of a frozen composition (Y(t+dt) = Y(t))
    for scale.  With mech_json, also the element conservation of both results:
    the largest relative change over the cells of each element's moles per
    unit mass (the frozen composition conserves them exactly)."""
    import torch
    Ti, Yi = T.clone(), Y.clone()
    st, _ = integrate(mech, Ti, p, Yi, dt)
    Td, Yd = T.clone(), Y.clone()
    nfb, used, _ = dnn.infer(mech, Td, p, Yd, dt)
    ok = used == 0
    err_Y = (Yd - Yi).abs()[:, ok]
    frozen = (Y - Yi).abs()[:, ok]
    # coefficient of determination of the predicted change of F(Y) per species
    lam = 0.1
    bct = lambda a: (a.clamp(min=0.0) ** lam - 1.0) / lam  # noqa: E731
    du_t = (bct(Yi) - bct(Y))[:, ok]
    du_p = (bct(Yd) - bct(Y))[:, ok]
    var = du_t.var(dim=1)
    r2 = 1.0 - ((du_p - du_t) ** 2).mean(dim=1) / torch.where(var > 0, var, torch.ones_like(var))
    extra = {}
    if mech_json is not None:
        A = torch.tensor(element_matrix(mech_json), device=T.device)
        b0 = A @ Y[:, ok]
        den = torch.clamp(b0.abs(), min=1e-300)
        extra["element_imbalance_dnn"] = ((A @ (Yd[:, ok] - Y[:, ok])).abs() / den).max(dim=1).values.cpu().numpy()
        extra["element_imbalance_integrator"] = \
            ((A @ (Yi[:, ok] - Y[:, ok])).abs() / den).max(dim=1).values.cpu().numpy()
    return {
        **extra,
        "r2_dF": r2.cpu().numpy(), "var_dF": var.cpu().numpy(),
        "n": int(T.numel()), "n_network": int(ok.sum()), "n_fallback": int(nfb),
        "mae_Y": err_Y.mean(dim=1).cpu().numpy(), "max_Y": err_Y.max(dim=1).values.cpu().numpy(),
        "mae_T": float((Td - Ti).abs()[ok].mean()), "max_T": float((Td - Ti).abs()[ok].max()),
        "frozen_mae_Y": frozen.mean(dim=1).cpu().numpy(),
        "frozen_mae_T": float((T - Ti).abs()[ok].mean()),
    }


def heldout(m: Mechanism, mech_json: dict, dnn: Dnn, n_eval: int, n_steps: int, oor_frac: float,
            seed: int = synth.TRAIN_SEED):
    """Held-out inference states: all time levels of integrator trajectories
    other than the training ones, with a fraction oor_frac moved outside the
    network's training T range (half 50-300 K below it, half 50-300 K above).
    Returns device tensors T, p, Y and the number of moved cells."""
    import torch
    n_init = max(1, n_eval // n_steps)
    Ts, p, Ys = trajectories(m, mech_json, n_init, n_steps - 1, seed=seed + 1000)
    Te = torch.cat(Ts)[:n_eval].contiguous()
    Pe = p.repeat(n_steps)[:n_eval].contiguous()
    Ye = torch.cat(Ys, dim=1)[:, :n_eval].contiguous()
    del Ts, Ys
    n_eval = Te.numel()
    g = torch.Generator(device=Te.device).manual_seed(seed + 7)
    n_oor = int(round(oor_frac * n_eval))
    oor = torch.randperm(n_eval, device=Te.device, generator=g)[:n_oor]
    nm = dnn.norm()
    t_lo, t_hi = float(nm["in_min"][0]), float(nm["in_max"][0])
    off = 50.0 + 250.0 * torch.rand(n_oor, device=Te.device, generator=g, dtype=torch.float64)
    half = n_oor // 2
    Te[oor[:half]] = t_lo - off[:half]
    Te[oor[half:]] = t_hi + off[half:]
    return Te, Pe, Ye, n_oor


def experiment(mech_json: dict, n_train_init=1 << 16, n_steps=32, n_eval=1 << 22, oor_frac=0.02,
               train_seconds=60.0, batch=4096, reps=3, seed=synth.TRAIN_SEED, log=None):
    """Learned-surrogate workload: train on integrator trajectories of the
    uneven-stiffness field, then advance n_eval held-out trajectory states (with
    a fraction moved above the training temperature range) by the network and,
    for comparison, by the integrator.  Returns throughput and error figures."""
    import torch

    def ev_time(fn, reps):
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            fn(e0, e1)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2]

    m = Mechanism(mech_json)
    t0 = time.time()
    Ts, p, Ys = trajectories(m, mech_json, n_train_init, n_steps, seed=seed)
    T0, P0, Y0, T1, Y1 = pairs(Ts, p, Ys)
    del Ts, Ys
    t_data = time.time() - t0
    o = dnn_default_opts()
    o.batch = batch
    dnn = Dnn(o, seed=seed)
    dnn.fit_norm(T0, P0, Y0, Y1)
    t1 = time.time()
    losses = train(dnn, T0, P0, Y0, Y1, epochs=10_000, batch=batch, time_budget=train_seconds, log=log)
    t_train = time.time() - t1
    n_pairs = T0.numel()
    del T0, P0, Y0, T1, Y1
    Te, Pe, Ye, n_oor = heldout(m, mech_json, dnn, n_eval, n_steps, oor_frac, seed)
    n_eval = Te.numel()
    # accuracy: network vs integrator on the same states
    ev = evaluate(dnn, m, Te, Pe, Ye, mech_json=mech_json)
    bound = within_bound(ev, inert_mask(mech_json))
    # throughput: network (incl. pre/post and fallback) and integrator, same cells
    Tw, Yw = Te.clone(), Ye.clone()

    def run_dnn(e0, e1):
        Tw.copy_(Te)
        Yw.copy_(Ye)
        e0.record()
        dnn.infer(m, Tw, Pe, Yw, 1e-6)
        e1.record()

    def run_int(e0, e1):
        Tw.copy_(Te)
        Yw.copy_(Ye)
        e0.record()
        integrate(m, Tw, Pe, Yw, 1e-6)
        e1.record()

    run_dnn(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))  # warm-up
    ms_dnn = ev_time(run_dnn, reps)
    ms_int = ev_time(run_int, reps)
    acc, rej = m.last_stats()
    r2 = ev["r2_dF"][ev["var_dF"] > 0]
    # the same pass split into the cells the network takes and the fallback
    # cells: how the time divides, and the bound the FP64 fallback sets on the
    # speed-up (the integrator's time over its time on the fallback cells alone)
    Tw.copy_(Te)
    Yw.copy_(Ye)
    _, used, _ = dnn.infer(m, Tw, Pe, Yw, 1e-6)
    split = {}
    for name, sel in (("network_cells_only", used == 0), ("fallback_cells_only", used != 0)):
        idx = sel.nonzero().squeeze(1)
        Ts, Ps, Ys = Te[idx].contiguous(), Pe[idx].contiguous(), Ye[:, idx].contiguous()
        Tx, Yx = Ts.clone(), Ys.clone()

        def run_d(e0, e1, Ts=Ts, Ps=Ps, Ys=Ys, Tx=Tx, Yx=Yx):
            Tx.copy_(Ts)
            Yx.copy_(Ys)
            e0.record()
            dnn.infer(m, Tx, Ps, Yx, 1e-6)
            e1.record()

        def run_i(e0, e1, Ts=Ts, Ps=Ps, Ys=Ys, Tx=Tx, Yx=Yx):
            Tx.copy_(Ts)
            Yx.copy_(Ys)
            e0.record()
            integrate(m, Tx, Ps, Yx, 1e-6)
            e1.record()

        ms_i = ev_time(run_i, reps)
        split[name] = {"cells": int(idx.numel()), "ms_integrator": ms_i}
        if name == "network_cells_only":
            ms_d = ev_time(run_d, reps)
            split[name].update({"ms_infer": ms_d, "infer_cells_per_s": idx.numel() / (ms_d * 1e-3),
                                "speedup_vs_integrator": ms_i / ms_d})
        else:
            split[name].update({"share_of_integrator_time_on_all_cells": ms_i / ms_int,
                                "speedup_bound_with_an_instant_network": ms_int / ms_i})
    return {
        "workload": f"train on {n_pairs} integrator pairs ({n_train_init} trajectories x {n_steps} steps of "
                    f"dt=1us); infer {n_eval} held-out trajectory states, {n_oor} moved outside the training "
                    f"T range (half below, half above)",
        "train": {"seconds": t_train, "steps": losses[-1][0] + 1 if losses else 0, "batch": batch,
                  "loss_first": losses[0][1] if losses else None, "loss_last": losses[-1][1] if losses else None,
                  "data_seconds": t_data},
        "infer_cells_per_s": n_eval / (ms_dnn * 1e-3),
        "integrator_cells_per_s": n_eval / (ms_int * 1e-3),
        "speedup_vs_integrator": ms_int / ms_dnn,
        "ms_infer": ms_dnn, "ms_integrator": ms_int,
        "n_fallback": ev["n_fallback"], "n_injected_out_of_range": n_oor,
        "error_vs_integrator": {
            "mae_Y_per_species": [float(x) for x in ev["mae_Y"]],
            "max_Y_per_species": [float(x) for x in ev["max_Y"]],
            "mae_T_K": ev["mae_T"], "max_T_K": ev["max_T"],
            "r2_dF_mean_reacting": float(np.mean(r2)) if r2.size else None,
            "frozen_composition_mae_Y": [float(x) for x in ev["frozen_mae_Y"]],
            "frozen_composition_mae_T_K": ev["frozen_mae_T"],
            "bound": bound,
            "element_imbalance_max_rel": {
                "dnn": [float(x) for x in ev["element_imbalance_dnn"]],
                "integrator": [float(x) for x in ev["element_imbalance_integrator"]],
                "frozen_composition": 0.0,
                "elements": sorted({e for sp in mech_json["species"] for e in sp["composition"]})},
        },
        "integrator_substeps_per_cell": (acc + rej) / n_eval,
        **split,
    }
