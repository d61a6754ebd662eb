"""Degenerate and boundary inputs through the C ABI, against closed forms or the oracle: a
single edge, an empty query list, only u == v queries, a star grounded at its centre (the
reduced graph falls apart into single nodes, so every leaf pair walks two branches ending in
different roots), a long chain (a deep etree), ragged grid sizes, and all three routes (walk,
block inverse, selected inverse) on each."""
import numpy as np
import pytest

from paper_2606_31535_b300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_31535_b300 import build, peers
    build.build()
    peers.load()
    return peers


@pytest.fixture(scope="module")
def ctx(P):
    return P.Context(0)


def routes(P, ctx, g, qu=None, qv=None, ground=0, use_coords=True, selinv=True):
    sym = P.Symbolic.of(g, ground, qu, qv, use_coords)
    num = P.Numeric(ctx, sym)
    out = [P.query(ctx, sym, num), P.query_blockinv(ctx, sym, num)]
    if selinv:
        out.append(P.query_selinv(ctx, sym, num))
    return out


def test_single_edge(P, ctx):
    g = I.from_edges(2, np.array([0]), np.array([1]), np.array([4.0]))
    for ground in (0, 1):
        for R in routes(P, ctx, g, ground=ground, use_coords=False):
            assert R.shape == (1,) and abs(R[0] - 0.25) < 1e-15


def test_empty_and_trivial_query_lists(P, ctx):
    g = I.grid2d(6, 7, seed=1)
    e = np.zeros(0, dtype=np.int32)
    for R in routes(P, ctx, g, e, e):
        assert R.shape == (0,)
    same = np.arange(10, dtype=np.int32)
    for R in routes(P, ctx, g, same, same):
        assert np.all(R == 0.0)


def test_star_grounded_at_its_centre(P, ctx):
    n = 40
    w = 10.0 ** np.random.default_rng(2).uniform(-2, 2, n - 1)
    g = I.from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n), w)
    leaf_u = np.array([1, 2, 5, 39, 7], dtype=np.int32)
    leaf_v = np.array([2, 3, 9, 1, 7], dtype=np.int32)
    qu = np.concatenate([np.zeros(n - 1, np.int32), leaf_u])
    qv = np.concatenate([np.arange(1, n, dtype=np.int32), leaf_v])
    expect = np.concatenate([1.0 / w, 1.0 / w[leaf_u - 1] + 1.0 / w[leaf_v - 1]])
    expect[-1] = 0.0   # (7, 7)
    # pairs of leaves lie outside the pattern of L: walk and block inverse only
    for R in routes(P, ctx, g, qu, qv, ground=0, use_coords=False, selinv=False):
        nz = expect != 0
        assert np.max(np.abs(R[nz] - expect[nz]) / expect[nz]) <= 1e-13
        assert R[-1] == 0.0
    # the edges alone through all three routes, grounded at a leaf instead
    for R in routes(P, ctx, g, ground=5, use_coords=False):
        assert np.max(np.abs(R - 1.0 / w) * w) <= 1e-13


def test_long_chain(P, ctx, oracle_mod):
    """A 3000-node path: the etree is one chain, and R_uv is the sum of 1/w between u and v
    (summed exactly).  Grounded at an end, L_r has condition number ~ n^2 ~ 1e7, so every
    LDL^T route carries rounding of order kappa * eps ~ 1e-9 at worst; 1e-10 holds with room."""
    import math
    n = 3000
    w = np.random.default_rng(3).uniform(0.5, 2.0, n - 1)
    g = I.from_edges(n, np.arange(n - 1), np.arange(1, n), w)
    pu, pv = I.random_pairs(n, 200, seed=4)
    r = 1.0 / w
    exact = np.array([math.fsum(r[min(a, b):max(a, b)]) for a, b in zip(pu, pv)])
    for ground in (0, 1500):
        Ro = oracle_mod.resistance(g, pu, pv, ground=ground, use_coords=False)
        assert np.max(np.abs(Ro - exact) / exact) < 1e-10
        for R in routes(P, ctx, g, pu, pv, ground=ground, use_coords=False, selinv=False):
            assert np.max(np.abs(R - Ro) / Ro) <= TOL
            assert np.max(np.abs(R - exact) / exact) < 1e-10
        for R in routes(P, ctx, g, ground=ground, use_coords=False):
            assert np.max(np.abs(R - r) * w) < 1e-10


@pytest.mark.parametrize("rows,cols", [(1, 57), (2, 2), (33, 65), (65, 33), (97, 31)])
def test_ragged_grids(P, ctx, oracle_mod, rows, cols):
    g = I.grid2d(rows, cols, seed=5 + rows, law="loguniform", lo=1e-3, hi=1e3)
    u, v = g.all_edges()
    Ro = oracle_mod.resistance(g, u, v)
    for R in routes(P, ctx, g):
        assert np.max(np.abs(R - Ro) / Ro) <= TOL
    assert abs(np.sum(g.edge_weights() * Ro) / (g.n - 1) - 1) < 1e-11
