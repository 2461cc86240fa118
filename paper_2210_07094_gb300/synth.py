"""Seeded synthetic inputs: reaction mechanisms and cell fields.

This module only *draws* inputs. It holds none of the chemistry the
integrator or the oracle evaluates (no rates, no Jacobian, no ODE); both the
CUDA path and the CPU oracle read what it writes.  Every draw comes from
``numpy.random.Generator(PCG64(seed))`` so a (recipe, seed) pair fixes the
bytes.

The paper's own workloads (0D constant-pressure H2/air ignition, Sec. 4.1;
DNN vs CVODE timing, Sec. 5.1) use the Evans H2 mechanism, which is not
available; the seeded mechanisms below stand in for it:

* ``h2_air_mechanism``: 9 species (H2 O2 H2O H O OH HO2 H2O2 N2, N2 inert),
  25 random reversible H/O-conserving reactions, 4 third-body and 2 Troe.
* ``hydrocarbon_mechanism``: 50 CHON species, 300 reactions, 20 third-body
  and 10 Troe.

The reaction set follows the reaction-system notation of Sec. 2.3 (eq. for
the reaction system): each reaction j lists nu'_{aj} (reactants) and
nu''_{aj} (products) over species a.

Units written to the mechanism JSON: A in cm, mol, s (order n counts M for
third-body reactions; Troe k0 is one order above k_inf), Ea in kJ/mol,
NASA-7 coefficients over one range 300-3000 K with a4 = a5 = 0.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import numpy as np

MECH_SEED = 7094
FIELD_SEED = 2210
TRAIN_SEED = 22

ATOMIC_MASS = {"H": 1.008, "C": 12.011, "N": 14.007, "O": 15.999}
P_ATM = 101325.0  # Pa
_R_GAS = 8.314462618  # J/(mol K); used only to place a6/a7 from drawn H_f, S


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _mol_weight(comp: dict) -> float:
    return float(sum(ATOMIC_MASS[e] * c for e, c in comp.items()))


def _formula(comp: dict) -> str:
    s = ""
    for e in ("C", "H", "O", "N"):
        c = comp.get(e, 0)
        if c == 1:
            s += e
        elif c > 1:
            s += f"{e}{c}"
    return s


def _draw_nasa7(rng, hf_kj: float, s_r: float, monatomic: bool) -> list:
    """Draw cp/R = a1 + a2 T + a3 T^2 positive on [300, 3000] K, then place a6
    and a7 so that H(298.15) = hf_kj and S(298.15)/R = s_r."""
    grid = np.arange(300.0, 3001.0, 1.0)
    while True:
        if monatomic:
            a1, a2, a3 = 2.5, 0.0, 0.0
        else:
            a1 = rng.uniform(2.5, 4.5)
            a2 = rng.uniform(0.0, 2e-3)
            a3 = rng.uniform(-3e-7, 0.0)
        if np.all(a1 + a2 * grid + a3 * grid * grid > 0.0):
            break
    t0 = 298.15
    # H/R at t0 from the cp/R polynomial integrated from 0, plus a6
    a6 = hf_kj * 1e3 / _R_GAS - (a1 * t0 + a2 * t0 ** 2 / 2 + a3 * t0 ** 3 / 3)
    a7 = s_r - (a1 * math.log(t0) + a2 * t0 + a3 * t0 ** 2 / 2)
    return [a1, a2, a3, 0.0, 0.0, a6, a7]


# ---------------------------------------------------------------------------
# reaction-set sampling
# ---------------------------------------------------------------------------

def _elem_vec(ms, comps, elements):
    v = [0] * len(elements)
    for s in ms:
        for i, e in enumerate(elements):
            v[i] += comps[s].get(e, 0)
    return tuple(v)


def _sample_reactions(rng, names, comps, elements, reactive, M, n_tb, n_troe):
    """Pick M distinct element-conserving reactions between multisets of 1-3
    reactive species.  The first n_tb + n_troe come from 1<->2 molecularity
    pairs (A + B <=> AB) so they can carry a third body or a falloff."""
    buckets: dict = {}
    for size in (1, 2, 3):
        for ms in itertools.combinations_with_replacement(reactive, size):
            buckets.setdefault(_elem_vec(ms, comps, elements), []).append(ms)
    multi = [k for k in sorted(buckets) if len(buckets[k]) >= 2]
    assoc = []
    for k in multi:
        ones = [m for m in buckets[k] if len(m) == 1]
        twos = [m for m in buckets[k] if len(m) == 2]
        assoc += [(a, b) for a in ones for b in twos]
    if len(assoc) < n_tb + n_troe:
        raise ValueError("not enough association pairs for third-body/Troe reactions")

    for _attempt in range(1000):
        chosen = []
        keys = set()

        def add(r, p):
            key = frozenset([r, p])
            if r == p or key in keys:
                return False
            keys.add(key)
            chosen.append((r, p))
            return True

        order = rng.permutation(len(assoc))
        kinds = []
        for idx in order:
            if len(chosen) == n_tb + n_troe:
                break
            a, b = assoc[idx]
            r, p = (a, b) if rng.random() < 0.5 else (b, a)
            if add(r, p):
                kinds.append("three-body" if len(kinds) < n_tb else "falloff-troe")
        # cover every reactive species at least once
        for s in rng.permutation(reactive):
            s = int(s)
            if any(s in r or s in p for r, p in chosen):
                continue
            cands = [(k, m) for k in multi for m in buckets[k] if s in m]
            k, m = cands[rng.integers(len(cands))]
            others = [o for o in buckets[k] if o != m]
            o = others[rng.integers(len(others))]
            r, p = (m, o) if rng.random() < 0.5 else (o, m)
            if add(r, p):
                kinds.append("elementary")
        while len(chosen) < M:
            k = multi[rng.integers(len(multi))]
            i, j = rng.choice(len(buckets[k]), size=2, replace=False)
            if add(buckets[k][i], buckets[k][j]):
                kinds.append("elementary")
        if len(chosen) != M:
            continue
        covered = set()
        for r, p in chosen:
            covered.update(r)
            covered.update(p)
        if covered >= set(reactive):
            return chosen, kinds
    raise RuntimeError("reaction sampling did not converge")


def _side(ms, names):
    d: dict = {}
    for s in ms:
        d[names[s]] = d.get(names[s], 0) + 1
    return d


def _side_str(d):
    parts = []
    for k, v in d.items():
        parts.append(k if v == 1 else f"{v} {k}")
    return " + ".join(parts)


def _build_mechanism(rng, name, names, comps, elements, hf, s_r, reactive,
                     M, n_tb, n_troe, seed, recipe):
    species = []
    for i, n in enumerate(names):
        natoms = sum(comps[n].values())
        species.append({
            "name": n,
            "composition": comps[n],
            "W": _mol_weight(comps[n]),
            "nasa7": _draw_nasa7(rng, hf[n], s_r[n], monatomic=(natoms == 1)),
            "T_range": [300.0, 3000.0],
            "Hf298": hf[n],
            "S298_R": s_r[n],
        })
    idx = [names.index(n) for n in reactive]
    comp_list = [comps[n] for n in names]
    chosen, kinds = _sample_reactions(rng, names, comp_list, elements, idx, M, n_tb, n_troe)
    reactions = []
    for (r, p), kind in zip(chosen, kinds):
        # write each reaction in its exothermic direction at 298 K, so the reverse
        # rate K_f/K_c carries an activation energy of at least Ea (a reaction drawn
        # endothermic with Ea < dH would get a reverse rate with a negative
        # activation energy of hundreds of kJ/mol)
        dh = sum(hf[names[k]] for k in p) - sum(hf[names[k]] for k in r)
        if dh > 0.0:
            r, p = p, r
        rd, pd = _side(r, names), _side(p, names)
        rxn = {
            "reactants": rd,
            "products": pd,
            "type": kind,
            "reversible": True,
            "A": float(10.0 ** rng.uniform(10.0, 16.0)),
            "b": float(rng.uniform(-1.5, 1.5)),
            "Ea": float(rng.uniform(0.0, 200.0)),
        }
        m_tag = ""
        if kind != "elementary":
            eff = {}
            for n in names:
                if rng.random() < 0.3:
                    eff[n] = float(rng.uniform(0.5, 12.0))
            rxn["efficiencies"] = eff
            m_tag = " + M" if kind == "three-body" else " (+M)"
        if kind == "falloff-troe":
            rxn["low"] = {"A": rxn["A"] * float(10.0 ** rng.uniform(3.0, 6.0)),
                          "b": rxn["b"], "Ea": rxn["Ea"]}
            rxn["troe"] = {"alpha": float(rng.uniform(0.1, 0.9)),
                           "T3": float(rng.uniform(30.0, 300.0)),
                           "T1": float(rng.uniform(500.0, 5000.0)),
                           "T2": float(rng.uniform(2000.0, 8000.0))}
        rxn["equation"] = f"{_side_str(rd)}{m_tag} <=> {_side_str(pd)}{m_tag}"
        reactions.append(rxn)
    return {
        "name": name,
        "generator": {"seed": seed, "recipe": recipe},
        "elements": elements,
        "units": {"A": "cm, mol, s", "Ea": "kJ/mol", "T": "K",
                  "nasa7": "cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4; one range"},
        "species": species,
        "reactions": reactions,
    }


H2_SPECIES = ["H2", "O2", "H2O", "H", "O", "OH", "HO2", "H2O2", "N2"]
_H2_COMP = {"H2": {"H": 2}, "O2": {"O": 2}, "H2O": {"H": 2, "O": 1}, "H": {"H": 1},
            "O": {"O": 1}, "OH": {"H": 1, "O": 1}, "HO2": {"H": 1, "O": 2},
            "H2O2": {"H": 2, "O": 2}, "N2": {"N": 2}}
# heats of formation at 298 K (kJ/mol): ranges drawn around water chemistry
_H2_HF = {"H2": (0, 0), "O2": (0, 0), "N2": (0, 0), "H2O": (-250, -230),
          "H2O2": (-145, -130), "HO2": (0, 20), "OH": (30, 45), "O": (240, 255),
          "H": (210, 225)}

# standard entropies S(298)/R: bands around those of the water-chemistry species
_H2_SR = {"H2": (15.0, 16.5), "O2": (24.0, 25.5), "H2O": (22.0, 23.5), "H": (13.0, 14.5),
          "O": (19.0, 20.5), "OH": (21.5, 23.0), "HO2": (26.5, 28.0), "H2O2": (27.5, 29.0),
          "N2": (22.5, 24.0)}


def _sr_band(comp: dict):
    """S(298)/R band that grows with the atom count (about 18 + 1.3 per atom)."""
    na = sum(comp.values())
    return (16.0 + 1.3 * na, 19.0 + 1.3 * na)


def h2_air_mechanism(seed: int = MECH_SEED, M: int = 25, n_tb: int = 4, n_troe: int = 2) -> dict:
    """9-species H2/air-like mechanism (N2 inert, collider only)."""
    rng = _rng(seed)
    hf = {n: float(rng.uniform(*_H2_HF[n])) if _H2_HF[n] != (0, 0) else 0.0 for n in H2_SPECIES}
    s_r = {n: float(rng.uniform(*_H2_SR[n])) for n in H2_SPECIES}
    reactive = [n for n in H2_SPECIES if n != "N2"]
    return _build_mechanism(rng, f"synthetic-h2air-{len(H2_SPECIES)}sp-{M}r", H2_SPECIES,
                            _H2_COMP, ["H", "O", "N"], hf, s_r, reactive, M, n_tb,
                            n_troe, seed, "h2_air_mechanism")


def hydrocarbon_mechanism(seed: int = MECH_SEED, n_species: int = 50, M: int = 300,
                          n_tb: int = 20, n_troe: int = 10) -> dict:
    """50-species CHON mechanism with 1-3 C_xH_y fuels."""
    rng = _rng(seed + 1)
    base = dict(_H2_COMP)
    base["CO"] = {"C": 1, "O": 1}
    base["CO2"] = {"C": 1, "O": 2}
    names = list(base)
    comps = dict(base)
    seen = {tuple(sorted(c.items())) for c in comps.values()}
    n_fuel = int(rng.integers(1, 4))
    fuels = []
    while len(fuels) < n_fuel:
        x = int(rng.integers(1, 5))
        y = int(rng.integers(2, 2 * x + 3))
        c = {"C": x, "H": y}
        key = tuple(sorted(c.items()))
        if key in seen:
            continue
        seen.add(key)
        n = _formula(c)
        names.append(n)
        comps[n] = c
        fuels.append(n)
    while len(names) < n_species:
        c = {"C": int(rng.integers(0, 4)), "H": int(rng.integers(0, 9)),
             "O": int(rng.integers(0, 4)), "N": int(rng.integers(0, 3))}
        c = {k: v for k, v in c.items() if v > 0}
        if not c or sum(c.values()) > 8 or sum(c.values()) < 2:
            continue
        key = tuple(sorted(c.items()))
        if key in seen:
            continue
        seen.add(key)
        n = _formula(c)
        names.append(n)
        comps[n] = c
    hf = {}
    for n in names:
        if n in _H2_HF:
            lo, hi = _H2_HF[n]
            hf[n] = float(rng.uniform(lo, hi)) if (lo, hi) != (0, 0) else 0.0
        elif n == "CO":
            hf[n] = float(rng.uniform(-115.0, -105.0))
        elif n == "CO2":
            hf[n] = float(rng.uniform(-400.0, -385.0))
        else:
            hf[n] = float(rng.uniform(-400.0, 300.0))
    s_r = {n: float(rng.uniform(*(_H2_SR[n] if n in _H2_SR else _sr_band(comps[n]))))
           for n in names}
    mech = _build_mechanism(rng, f"synthetic-chon-{n_species}sp-{M}r", names, comps,
                            ["C", "H", "O", "N"], hf, s_r, names, M, n_tb, n_troe,
                            seed, "hydrocarbon_mechanism")
    mech["fuels"] = fuels
    return mech


# ---------------------------------------------------------------------------
# small mechanisms with closed-form behaviour (test inputs)
# ---------------------------------------------------------------------------

def _iso_species(a7_b: float, W: float = 30.0):
    nasa = [3.5, 1e-3, -1e-7, 0.0, 0.0, -1000.0, 10.0]
    nb = list(nasa)
    nb[6] = a7_b
    return [
        {"name": "A", "composition": {"X": 2}, "W": W, "nasa7": nasa, "T_range": [300.0, 3000.0]},
        {"name": "B", "composition": {"X": 2}, "W": W, "nasa7": nb, "T_range": [300.0, 3000.0]},
        {"name": "D", "composition": {"Z": 1}, "W": W, "nasa7": [2.5, 0, 0, 0, 0, -745.375, 4.0],
         "T_range": [300.0, 3000.0]},
    ]


def isomer_mechanism(kind: str = "elementary", A: float = 2.0e5, b: float = 0.0,
                     Ea: float = 0.0, a7_b: float = 10.7, reversible: bool = True,
                     eff: dict | None = None, low: dict | None = None,
                     troe: dict | None = None) -> dict:
    """A <=> B (+ inert D) between isomers of equal W and equal enthalpy.

    Because A and B have the same cp and h, dT/dt = 0 and the problem is a
    linear two-state decay with a closed-form solution.  ``a7_b`` sets
    K_c = exp(a7_B - a7_A).
    """
    rxn = {"reactants": {"A": 1}, "products": {"B": 1}, "type": kind,
           "reversible": reversible, "A": A, "b": b, "Ea": Ea, "equation": "A <=> B"}
    if kind != "elementary":
        rxn["efficiencies"] = dict(eff or {})
    if kind == "falloff-troe":
        rxn["low"] = dict(low)
        rxn["troe"] = dict(troe)
    return {"name": f"isomer-{kind}", "elements": ["X", "Z"],
            "units": {"A": "cm, mol, s", "Ea": "kJ/mol", "T": "K"},
            "species": _iso_species(a7_b), "reactions": [rxn]}


def autocatalytic_mechanism(A: float = 1.0e7, da6: float = -1.0, W: float = 30.0) -> dict:
    """A + B -> 2 B (irreversible, b = 0, Ea = 0) with an inert D; A, B and D
    have the same W and cp, and B's enthalpy sits da6 * R below A's.  At
    constant pressure with W-bar fixed, dY_B/dt = r Y_A Y_B, r = A rho / W (a
    logistic curve), and dT/dt is proportional to the same product: the rate
    peaks where Y_A = Y_B.  With |da6| small the temperature (and rho) barely
    moves, so the time of [dT/dt]_max is ln(Y_A0 / Y_B0) / (r (Y_A0 + Y_B0))."""
    base = [3.5, 1e-3, -1e-7, 0.0, 0.0, -1000.0, 10.0]
    nb = list(base)
    nb[5] = base[5] + da6
    sp = [{"name": "A", "composition": {"X": 2}, "W": W, "nasa7": base, "T_range": [300.0, 3000.0]},
          {"name": "B", "composition": {"X": 2}, "W": W, "nasa7": nb, "T_range": [300.0, 3000.0]},
          {"name": "D", "composition": {"Z": 1}, "W": W, "nasa7": list(base), "T_range": [300.0, 3000.0]}]
    rxn = {"reactants": {"A": 1, "B": 1}, "products": {"B": 2}, "type": "elementary", "reversible": False,
           "A": A, "b": 0.0, "Ea": 0.0, "equation": "A + B => 2 B"}
    return {"name": "autocatalytic", "elements": ["X", "Z"], "units": {"A": "cm, mol, s", "Ea": "kJ/mol", "T": "K"},
            "species": sp, "reactions": [rxn]}


def zero_rate(mech: dict) -> dict:
    """Same species and reactions with every pre-exponential set to 0."""
    m = json.loads(json.dumps(mech))
    for r in m["reactions"]:
        r["A"] = 0.0
        if "low" in r:
            r["low"]["A"] = 0.0
    m["name"] = mech["name"] + "-zero-rate"
    return m


# ---------------------------------------------------------------------------
# cell fields (species-major SoA: Y[k][c])
# ---------------------------------------------------------------------------

def _h2_air_Y(mech, phi):
    names = [s["name"] for s in mech["species"]]
    W = {s["name"]: s["W"] for s in mech["species"]}
    n = phi.shape[0]
    Y = np.zeros((len(names), n))
    rad = ["H", "O", "OH", "HO2", "H2O2"]
    m_h2 = 2.0 * phi * W["H2"]
    m_o2 = np.full(n, 1.0 * W["O2"])
    m_n2 = np.full(n, 3.76 * W["N2"])
    tot = m_h2 + m_o2 + m_n2
    scale = 1.0 - 1e-6 * len(rad)
    Y[names.index("H2")] = m_h2 / tot * scale
    Y[names.index("O2")] = m_o2 / tot * scale
    Y[names.index("N2")] = m_n2 / tot * scale
    for r in rad:
        Y[names.index(r)] = 1e-6
    return Y


def _fuel_air_Y(mech, phi, rng):
    names = [s["name"] for s in mech["species"]]
    comp = {s["name"]: s["composition"] for s in mech["species"]}
    W = np.array([s["W"] for s in mech["species"]])
    fuels = mech["fuels"]
    n = phi.shape[0]
    X = np.zeros((len(names), n))
    fx = rng.dirichlet(np.ones(len(fuels)), size=n).T  # fuel mole split
    o2_per_fuel = np.zeros(n)
    for i, f in enumerate(fuels):
        c = comp[f]
        o2_per_fuel += fx[i] * (c.get("C", 0) + c.get("H", 0) / 4.0 - c.get("O", 0) / 2.0)
        X[names.index(f)] = fx[i]
    n_o2 = o2_per_fuel / phi
    X[names.index("O2")] = n_o2
    X[names.index("N2")] = 3.76 * n_o2
    m = X * W[:, None]
    Y = m / m.sum(axis=0)
    major = set(fuels) | {"O2", "N2"}
    others = [i for i, s in enumerate(names) if s not in major]
    Y *= (1.0 - 1e-6 * len(others))
    Y[others] = 1e-6
    return Y


# The synthetic workloads, by index: 0 the 9-species H2/air parity field (4096
# cells, 900-1500 K, 1 atm); 1 the uneven-stiffness field of the throughput
# benchmark (2^20 cells, half 700-1000 K and half 1800-2500 K interleaved,
# 1-10 atm); 2 the 50-species CHON field (262144 cells, 800-2200 K, 1 atm); 3
# the adjoint field (65536 cells, as 0); 4 the surrogate's field (2^22 cells,
# as 1).  dt = 1 us throughout.
CONFIGS = {
    0: dict(ncells=4096, T=("uniform", 900.0, 1500.0), p=("const", 1.0), mech="h2"),
    1: dict(ncells=1 << 20, T=("bimodal", 700.0, 1000.0, 1800.0, 2500.0), p=("uniform", 1.0, 10.0),
            mech="h2"),
    2: dict(ncells=262144, T=("uniform", 800.0, 2200.0), p=("const", 1.0), mech="chon"),
    3: dict(ncells=65536, T=("uniform", 900.0, 1500.0), p=("const", 1.0), mech="h2"),
    4: dict(ncells=1 << 22, T=("bimodal", 700.0, 1000.0, 1800.0, 2500.0), p=("uniform", 1.0, 10.0),
            mech="h2"),
}
DT = 1e-6


def mechanism_for(cfg: int) -> dict:
    return hydrocarbon_mechanism() if CONFIGS[cfg]["mech"] == "chon" else h2_air_mechanism()


def field(cfg: int, mech: dict, ncells: int | None = None, seed: int | None = None) -> dict:
    """Initial cell states of a config: T [K], p [Pa], Y[k][c] (species-major)."""
    c = CONFIGS[cfg]
    n = c["ncells"] if ncells is None else int(ncells)
    rng = _rng(FIELD_SEED + cfg if seed is None else seed)
    tk = c["T"]
    if tk[0] == "uniform":
        T = rng.uniform(tk[1], tk[2], n)
    else:
        hot = np.zeros(n, dtype=bool)
        hot[rng.permutation(n)[: n // 2]] = True
        T = np.where(hot, rng.uniform(tk[3], tk[4], n), rng.uniform(tk[1], tk[2], n))
    pk = c["p"]
    p = np.full(n, pk[1] * P_ATM) if pk[0] == "const" else rng.uniform(pk[1], pk[2], n) * P_ATM
    phi = rng.uniform(0.5, 2.0, n)
    Y = _fuel_air_Y(mech, phi, rng) if c["mech"] == "chon" else _h2_air_Y(mech, phi)
    return {"T": T, "p": p, "Y": np.ascontiguousarray(Y), "dt": DT}


def write_json(mech: dict, path: str) -> str:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        json.dump(mech, f, indent=1)
    return path
