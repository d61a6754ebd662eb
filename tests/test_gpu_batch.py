"""Batched sweep of many graphs (one persistent launch per aligned level, CUDA graph replay):
each graph's results equal its own single-graph sweep bit for bit, and the oracle."""
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


def small_batch():
    gs = []
    for i in range(10):
        if i % 2 == 0:
            r = 15 + 7 * i
            gs.append(I.grid_deleted(r, r + 3, seed=100 + i))
        else:
            gs.append(I.rgg(800 + 400 * i, seed=100 + i))
    return gs


@pytest.mark.parametrize("cuda_graph", [True, False])
def test_batch_equals_single_sweeps(P, oracle_mod, cuda_graph):
    gs = small_batch()
    ctx = P.Context(0)
    syms, nums, singles = [], [], []
    for i, g in enumerate(gs):
        if i == 3:   # one graph with listed pairs, including two-branch ones
            pu, pv = I.random_pairs(g.n, 400, seed=7)
            s = P.Symbolic.of(g, 0, pu, pv)
        elif i == 4:   # and one with many waves
            opt = P.Options()
            opt.carry_budget = 128 * 1024
            s = P.Symbolic.of(g, options=opt)
        else:
            s = P.Symbolic.of(g)
        m = P.Numeric(ctx, s)
        syms.append(s)
        nums.append(m)
        singles.append(P.query(ctx, s, m))
    b = P.Batch(ctx, syms, nums, cuda_graph=cuda_graph)
    info = b.info()
    assert info["launches"] < sum(s.info()["levels"] for s in syms)
    for rep in range(2):   # the second query replays the captured graph
        outs = b.query()
        for i in range(len(gs)):
            assert np.array_equal(outs[i], singles[i]), i
    for i in (0, 3, 5):
        g = gs[i]
        if i == 3:
            qu, qv = I.random_pairs(g.n, 400, seed=7)
        else:
            qu, qv = g.all_edges()
        Ro = oracle_mod.resistance(g, qu, qv)
        assert np.max(np.abs(outs[i] - Ro) / Ro) <= TOL


def test_batch_device_outputs(P):
    import torch
    gs = small_batch()[:4]
    ctx = P.Context(0)
    syms = [P.Symbolic.of(g) for g in gs]
    nums = [P.Numeric(ctx, s) for s in syms]
    b = P.Batch(ctx, syms, nums)
    outs = [torch.empty(s.nq, dtype=torch.float64, device="cuda:0") for s in syms]
    b.query(outs)
    torch.cuda.synchronize()
    for s, m, o in zip(syms, nums, outs):
        assert np.array_equal(o.cpu().numpy(), P.query(ctx, s, m))
