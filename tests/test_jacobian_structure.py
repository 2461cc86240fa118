"""Structure of the 50-species Jacobian: why the integrator keeps a dense LU.

A sparse analytic Jacobian with a sparse LU pays off only when the reaction
graph leaves most of d f / d y zero and the factorisation fills little of it
in.  On the 50-species / 300-reaction mechanism neither holds:

* at constant pressure C_k = rho Y_k / W_k with rho = p Wbar / (R T), so every
  rate depends on every mass fraction through the mean molar mass: the
  Jacobian of a real state has no zero entry at all (checked on the oracle's
  Jacobian);
* even without that coupling (the constant-volume closure), the 30 third-body
  and falloff reactions have a default efficiency of 1 for every species, so
  the rows of their 38 participating species are dense, and the reaction
  graph fills 97% of the matrix; eliminating it in degree order leaves the
  factorisation within 4% of the dense (2/3) n^3 flop count;
* splitting every dense part off as a low-rank update to be restored by
  Sherman-Morrison-Woodbury (the T row and column, the mean-molar-mass
  coupling, the unit part of the collider efficiencies) leaves a species
  block that the trimolecular reactions alone make 83% dense, which a
  minimum-degree elimination fills to 97%: its LU would save about 10% of the
  dense flops while the low-rank corrections add solves per stage.
"""
import numpy as np
import pytest

from oracle.oracle import Mech
from paper_2210_07094_gb300 import synth


@pytest.fixture(scope="module")
def chon():
    return synth.hydrocarbon_mechanism()


def _graph_pattern(mech):
    """Nonzero pattern of d f / d y implied by the reaction lists alone (T row
    and column dense; a reaction couples the species it changes to the species
    its rate depends on: its reactants and products, and every species when a
    collider [M] enters)."""
    names = [s["name"] for s in mech["species"]]
    idx = {n: i for i, n in enumerate(names)}
    N = len(names)
    n = N + 1
    P = np.zeros((n, n), dtype=bool)
    P[0, :] = True
    P[:, 0] = True
    np.fill_diagonal(P, True)
    for r in mech["reactions"]:
        nu = {}
        for k, v in r["reactants"].items():
            nu[idx[k]] = nu.get(idx[k], 0) - v
        for k, v in r["products"].items():
            nu[idx[k]] = nu.get(idx[k], 0) + v
        changed = [k for k, v in nu.items() if v != 0]
        deps = set(idx[k] for k in r["reactants"]) | set(idx[k] for k in r["products"])
        if r["type"] != "elementary":
            deps = set(range(N))
        for i in changed:
            for j in deps:
                P[1 + i, 1 + j] = True
    return P


def _lu_flops(P, order):
    """Multiply-adds (counted as 2 flop) and divisions of an LU without
    pivoting on the symbolic pattern P eliminated in the given order."""
    A = P[np.ix_(order, order)].copy()
    n = A.shape[0]
    flops = 0
    for k in range(n):
        rows = np.nonzero(A[k + 1:, k])[0] + k + 1
        cols = np.nonzero(A[k, k + 1:])[0] + k + 1
        flops += len(rows) + 2 * len(rows) * len(cols)
        for i in rows:
            A[i, cols] = True
    return flops


def test_constant_pressure_jacobian_has_no_zero_entry(chon):
    o = Mech(chon)
    f = synth.field(2, chon, 4, seed=3)
    for c in range(4):
        y = np.concatenate([[f["T"][c]], f["Y"][:, c]])
        J = o.jac(f["p"][c], y)
        assert J.shape == (51, 51)
        assert np.count_nonzero(J) == J.size


def test_reaction_graph_is_dense_and_sparse_lu_saves_little(chon):
    P = _graph_pattern(chon)
    n = P.shape[0]
    assert n == 51
    density = P.sum() / P.size
    assert density > 0.95, density
    dense = _lu_flops(np.ones_like(P), np.arange(n))
    # dense count is the textbook sum over k of (n-k-1) + 2 (n-k-1)^2
    assert dense == sum((n - k - 1) + 2 * (n - k - 1) ** 2 for k in range(n))
    deg = P.sum(axis=0) + P.sum(axis=1)
    order = np.concatenate([np.argsort(deg[1:], kind="stable") + 1, [0]])  # T last
    for perm in (np.arange(n), order):
        sparse = _lu_flops(P, perm)
        assert sparse > 0.95 * dense, (sparse, dense)


def test_pattern_helper_on_a_sparse_mechanism():
    """The pattern helper itself: an isomerisation A <=> B among otherwise
    inert species couples only A and B (plus the T row and column)."""
    mech = synth.isomer_mechanism()
    P = _graph_pattern(mech)
    n = P.shape[0]
    off = P.copy()
    off[0, :] = False
    off[:, 0] = False
    np.fill_diagonal(off, False)
    assert off.sum() == 2  # d f_A / d Y_B and d f_B / d Y_A
    # eliminated with T last the inert species creates no fill
    t_last = np.concatenate([np.arange(1, n), [0]])
    assert _lu_flops(P, t_last) < _lu_flops(np.ones_like(P), t_last)


def _species_pattern(mech):
    """Species block of the concentration-space Jacobian with every dense part
    split off: a reaction couples the species it changes to its reactants and
    products only (the collider sums and the mean-molar-mass coupling are
    rank-one terms, the T row and column a border)."""
    names = [s["name"] for s in mech["species"]]
    idx = {n: i for i, n in enumerate(names)}
    N = len(names)
    P = np.eye(N, dtype=bool)
    for r in mech["reactions"]:
        nu = {}
        for k, v in r["reactants"].items():
            nu[idx[k]] = nu.get(idx[k], 0) - v
        for k, v in r["products"].items():
            nu[idx[k]] = nu.get(idx[k], 0) + v
        deps = set(idx[k] for k in r["reactants"]) | set(idx[k] for k in r["products"])
        for i in (k for k, v in nu.items() if v != 0):
            for j in deps:
                P[i, j] = True
    return P


def _min_degree_order(P):
    """Greedy minimum-degree elimination order on the symmetrised pattern,
    with the fill of each elimination added to the graph."""
    G = P | P.T
    n = G.shape[0]
    alive = np.ones(n, dtype=bool)
    order = []
    for _ in range(n):
        deg = np.where(alive, (G & alive[None, :]).sum(axis=1), n + 1)
        k = int(np.argmin(deg))
        nb = np.nonzero(G[k] & alive)[0]
        nb = nb[nb != k]
        G[np.ix_(nb, nb)] = True
        alive[k] = False
        order.append(k)
    return np.array(order)


def test_species_block_stays_dense_with_the_dense_parts_split_off(chon):
    P = _species_pattern(chon)
    N = P.shape[0]
    assert N == 50
    assert P.sum() / P.size > 0.75
    order = _min_degree_order(P)
    sparse = _lu_flops(P, order)
    dense = _lu_flops(np.ones_like(P), np.arange(N))
    assert 0.85 * dense < sparse < dense, (sparse, dense)
