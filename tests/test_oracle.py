"""Pins for the CPU oracle against facts fixed by the mathematics, not by the oracle itself.

Each check would fail on a plausible slip in oracle.c: a dropped degree term (the edge to the
ground), a wrong sign in the triangular solve, a transposed factor, a missing path node, or a
wrong grounded case (eq. 4).
"""
import json
import os

import numpy as np
import pytest

from paper_2606_31535_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)) if a.size else 0.0


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "closed_forms.json")))["cases"],
                         ids=lambda c: c["name"])
@pytest.mark.parametrize("ground", [0, 3])
def test_golden_closed_forms(oracle_mod, case, ground):
    e = np.array(case["edges"], dtype=np.float64)
    g = I.from_edges(case["n"], e[:, 0].astype(np.int64), e[:, 1].astype(np.int64), e[:, 2])
    q = np.array(case["queries"], dtype=np.float64)
    R = oracle_mod.resistance(g, q[:, 0].astype(np.int32), q[:, 1].astype(np.int32),
                              ground=ground, use_coords=False)
    assert rel(R, q[:, 2]) < 1e-14


@pytest.mark.parametrize("maker", [
    lambda: I.grid2d(12, 13, seed=11),
    lambda: I.grid2d(9, 30, seed=12, law="loguniform", lo=1e-2, hi=1e2),
    lambda: I.pdn3(side=9, layers=3, via_stride=4, seed=13),
    lambda: I.grid_deleted(15, 17, seed=14),
    lambda: I.rgg(500, seed=15),
], ids=["grid", "grid-loguniform", "pdn3", "grid-deleted", "rgg"])
@pytest.mark.parametrize("use_coords", [True, False])
def test_against_dense_pseudoinverse(oracle_mod, maker, use_coords):
    g = maker()
    u, v = g.all_edges()
    pu, pv = I.random_pairs(g.n, 200, seed=99)
    qu = np.concatenate([u, pu])
    qv = np.concatenate([v, pv])
    R = oracle_mod.resistance(g, qu, qv, ground=0, use_coords=use_coords)
    Rd = oracle_mod.dense_resistance(g, qu, qv)
    # pinv of a Laplacian with conductances spanning 1e4 loses a few digits itself
    assert rel(R, Rd) < 1e-9


def test_tree_path_sums(oracle_mod):
    """On a tree every pair's resistance is the sum of 1/w along its unique path."""
    rng = np.random.default_rng(5)
    n = 300
    par = np.array([-1] + [int(rng.integers(0, i)) for i in range(1, n)])
    w = 10 ** rng.uniform(-2, 2, size=n)
    g = I.from_edges(n, np.arange(1, n), par[1:], w[1:])
    depth = np.zeros(n, dtype=int)
    for i in range(1, n):
        depth[i] = depth[par[i]] + 1

    def path_res(a, b):
        s = 0.0
        while a != b:
            if depth[a] >= depth[b]:
                s += 1.0 / w[a]
                a = par[a]
            else:
                s += 1.0 / w[b]
                b = par[b]
        return s

    qu, qv = I.random_pairs(n, 300, seed=6)
    R = oracle_mod.resistance(g, qu, qv, ground=17, use_coords=False)
    expect = np.array([path_res(int(a), int(b)) for a, b in zip(qu, qv)])
    assert rel(R, expect) < 1e-12
    eu, ev = g.all_edges()
    Re = oracle_mod.resistance(g, eu, ev, ground=0, use_coords=False)
    assert rel(Re, 1.0 / g.edge_weights()) < 1e-12


def test_cycle_closed_form(oracle_mod):
    """Cycle: edge e with resistance r_e in parallel with the rest of the loop, S - r_e."""
    rng = np.random.default_rng(7)
    n = 61
    w = rng.uniform(0.5, 2.0, size=n)
    g = I.from_edges(n, np.arange(n), (np.arange(n) + 1) % n, w)
    eu, ev = g.all_edges()
    Re = oracle_mod.resistance(g, eu, ev, ground=30, use_coords=False)
    r = 1.0 / g.edge_weights()
    S = np.sum(1.0 / w)
    assert rel(Re, r * (S - r) / S) < 1e-12


def test_complete_graph(oracle_mod):
    n = 40
    iu, iv = np.triu_indices(n, 1)
    g = I.from_edges(n, iu, iv, np.ones(iu.size))
    R = oracle_mod.resistance(g, iu, iv, ground=5, use_coords=False)
    assert rel(R, np.full(iu.size, 2.0 / n)) < 1e-12


@pytest.mark.parametrize("maker", [I.grid32, lambda: I.pdn3(side=33, seed=21),
                                   lambda: I.rgg(3000, seed=22)], ids=["grid32", "pdn3-33", "rgg"])
def test_foster(oracle_mod, maker):
    """Foster's theorem: sum over edges of w_e R_e = n - 1 for a connected graph."""
    g = maker()
    u, v = g.all_edges()
    R = oracle_mod.resistance(g, u, v)
    assert abs(np.sum(g.edge_weights() * R) / (g.n - 1) - 1.0) < 1e-11


def test_ground_invariance_and_grounded_queries(oracle_mod):
    g = I.grid2d(20, 21, seed=31, law="loguniform", lo=1e-2, hi=1e2)
    u, v = g.all_edges()
    pu, pv = I.random_pairs(g.n, 300, seed=32)
    # queries that touch node 0 and node 137 exercise the grounded cases of eq. 4
    extra_u = np.array([0, 5, 137, 0, 137], dtype=np.int32)
    extra_v = np.array([9, 0, 3, 137, 200], dtype=np.int32)
    qu = np.concatenate([u, pu, extra_u])
    qv = np.concatenate([v, pv, extra_v])
    R0 = oracle_mod.resistance(g, qu, qv, ground=0)
    R1 = oracle_mod.resistance(g, qu, qv, ground=137)
    Rd = oracle_mod.dense_resistance(g, qu, qv)
    assert rel(R0, R1) < 1e-10
    assert rel(R0, Rd) < 1e-9


def test_same_node_is_zero(oracle_mod):
    g = I.grid32()
    R = oracle_mod.resistance(g, np.array([3, 0, 77]), np.array([3, 0, 77]))
    assert np.all(R == 0.0)


def test_rayleigh_monotonicity(oracle_mod):
    """Raising one conductance can only lower effective resistances."""
    g = I.grid2d(14, 14, seed=41)
    qu, qv = I.random_pairs(g.n, 400, seed=42)
    R = oracle_mod.resistance(g, qu, qv)
    w2 = g.w.copy()
    rows = np.repeat(np.arange(g.n), np.diff(g.indptr))
    hit = ((rows == 50) & (g.indices == 51)) | ((rows == 51) & (g.indices == 50))
    w2[hit] *= 10.0
    g2 = I.Graph(g.n, g.indptr, g.indices, w2, g.coords)
    R2 = oracle_mod.resistance(g2, qu, qv)
    assert np.all(R2 <= R * (1 + 1e-12))
    assert np.any(R2 < R * (1 - 1e-6))


def test_triangle_inequality(oracle_mod):
    """Effective resistance is a metric on the nodes."""
    g = I.rgg(800, seed=51)
    rng = np.random.default_rng(52)
    a, b, c = (rng.integers(0, g.n, size=500) for _ in range(3))
    F = oracle_mod.Factor.of(g)
    Rab, Rbc, Rac = F.resistance(a, b), F.resistance(b, c), F.resistance(a, c)
    assert np.all(Rac <= (Rab + Rbc) * (1 + 1e-12))


def test_full_solve_identity_and_residual(oracle_mod):
    """sum_k y_k^2/d_k equals b^T x for x = L_r^{-1} b from a complete solve, and that x
    satisfies the unfactored system."""
    g = I.pdn3(side=25, seed=61)
    F = oracle_mod.Factor.of(g)
    u, v = g.all_edges()
    idx = np.random.default_rng(62).choice(u.size, 30, replace=False)
    R = F.resistance(u[idx], v[idx])
    for k, e in enumerate(idx):
        Rf, res = F.full_solve(int(u[e]), int(v[e]))
        assert abs(Rf - R[k]) <= 1e-11 * R[k]
        assert res < 1e-10


def test_elimination_tree_is_valid(oracle_mod):
    """Every etree parent is later in elimination order (Thm 1's ordering property)."""
    g = I.grid2d(17, 19, seed=71)
    F = oracle_mod.Factor.of(g)
    d, par, perm = F.export()
    k = np.arange(par.size)
    assert np.all((par == -1) | (par > k))
    assert np.all(d > 0)
    assert np.array_equal(np.sort(perm), np.arange(par.size))


def test_sparsifier_is_unbiased_and_preserves_the_quadratic_form(oracle_mod):
    """Alg. 1: every draw lands on an edge (counts sum to q), E[weight_e] = w_e, and the
    sparsifier's Laplacian approximates the graph's on random vectors."""
    g = I.grid2d(14, 15, seed=81, law="loguniform", lo=1e-2, hi=1e2)
    u, v = g.all_edges()
    w = g.edge_weights()
    R = oracle_mod.resistance(g, u, v)
    q = 400_000
    draws = np.random.default_rng(82).random(q)
    count, weight = oracle_mod.sparsify(w, R, q, draws)
    assert count.sum() == q
    # p_e ~ w_e R_e / (n - 1) by Foster; the heaviest edges are drawn near q p_e times
    p = w * R / np.sum(w * R)
    assert np.all(np.abs(count - q * p) <= 6 * np.sqrt(q * p) + 2)
    assert abs(weight.sum() / w.sum() - 1) < 0.05
    rng = np.random.default_rng(83)
    for _ in range(10):
        x = rng.standard_normal(g.n)
        full = np.sum(w * (x[u] - x[v]) ** 2)
        spars = np.sum(weight * (x[u] - x[v]) ** 2)
        assert 0.8 < spars / full < 1.2
