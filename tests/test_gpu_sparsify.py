"""Alg. 1 (spectral sparsification by effective resistances) on the device: the draws match
the oracle's sampler exactly on the same inputs, and the whole pipeline (resistances from the
sweep, then sparsification) preserves the Laplacian's quadratic form."""
import numpy as np
import pytest

from paper_2606_31535_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_31535_b300 import build, peers
    build.build()
    peers.load()
    return peers


def test_draws_match_the_oracle_sampler_exactly(P, oracle_mod):
    import torch
    g = I.pdn3(side=41, seed=90)
    u, v = g.all_edges()
    w = g.edge_weights()
    R = oracle_mod.resistance(g, u, v)
    q = 200_000
    draws = np.random.default_rng(91).random(q)
    c_ref, w_ref = oracle_mod.sparsify(w, R, q, draws)
    ctx = P.Context(0)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    count, weight = P.sparsify(ctx, dev(w), dev(R), dev(draws))
    torch.cuda.synchronize()
    assert np.array_equal(count.cpu().numpy(), c_ref)
    assert np.allclose(weight.cpu().numpy(), w_ref, rtol=1e-15, atol=0)


def test_sweep_then_sparsify_preserves_the_quadratic_form(P):
    import torch
    g = I.grid2d(40, 41, seed=92, law="loguniform", lo=1e-2, hi=1e2)
    u, v = g.all_edges()
    ctx = P.Context(0)
    sym = P.Symbolic.of(g)
    num = P.Numeric(ctx, sym)
    R = torch.empty(sym.nq, dtype=torch.float64, device="cuda:0")
    P.query(ctx, sym, num, R)
    w = torch.from_numpy(g.edge_weights()).cuda()
    q = 600_000
    draws = torch.from_numpy(np.random.default_rng(93).random(q)).cuda()
    count, weight = P.sparsify(ctx, w, R, draws)
    torch.cuda.synchronize()
    assert int(count.sum().item()) == q
    wt = weight.cpu().numpy()
    wn = g.edge_weights()
    kept = np.count_nonzero(wt)
    assert kept < wn.size              # a sparsifier drops edges
    rng = np.random.default_rng(94)
    for _ in range(10):
        x = rng.standard_normal(g.n)
        full = np.sum(wn * (x[u] - x[v]) ** 2)
        spars = np.sum(wt * (x[u] - x[v]) ** 2)
        assert 0.8 < spars / full < 1.2
