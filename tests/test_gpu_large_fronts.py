"""Supernode fronts larger than one CTA's shared memory (the sweep's spill path).

Nested dissection of large 2-D meshes, 3-D-like meshes and industrial graphs gives top
separators of many thousand rows, whose query fronts do not fit the 227 KiB of shared memory
of one CTA.  Such supernodes keep each tile's fronts in a global scratch slice of the CTA
that works on them; the operations, and so the results, stay the same bit for bit.  The
option peers_options.front_smem lowers the shared-memory budget so that graphs of test size
take that path: here every supernode (budget of 1 byte), and only the larger ones (8 KiB).
"""
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


def graph_and_queries(name):
    if name == "grid-200":
        g = I.grid2d(200, 200, seed=11, law="loguniform", lo=1e-3, hi=1e3)
        return g, None, None
    g = I.pdn3(side=49, seed=8)
    u, v = g.all_edges()
    pu, pv = I.random_pairs(g.n, 1500, seed=81)          # two-branch walks too
    return g, np.concatenate([u, pu]), np.concatenate([v, pv])


def sweep(P, ctx, g, qu, qv, front_smem=0):
    opt = P.Options()
    opt.front_smem = front_smem
    sym = P.Symbolic.of(g, 0, qu, qv, True, opt)
    num = P.Numeric(ctx, sym)
    return P.query(ctx, sym, num), sym


@pytest.mark.parametrize("name", ["grid-200", "pdn3-49"])
@pytest.mark.parametrize("front_smem", [1, 8 << 10])
def test_fronts_in_global_memory_match_shared_memory_bit_for_bit(P, oracle_mod, name,
                                                                  front_smem):
    ctx = P.Context(0)
    g, qu, qv = graph_and_queries(name)
    ref, sym0 = sweep(P, ctx, g, qu, qv)
    assert sym0.info()["nsuper_spilled"] == 0
    R, sym = sweep(P, ctx, g, qu, qv, front_smem)
    info = sym.info()
    assert info["nsuper_spilled"] > 0
    if front_smem == 1:
        assert info["nsuper_spilled"] == info["nsuper"]
    else:
        assert info["nsuper_spilled"] < info["nsuper"]
    assert info["walk_entries"] == sym0.info()["walk_entries"]
    assert np.array_equal(R, ref)
    if qu is None:
        qu, qv = g.all_edges()
    Ro = oracle_mod.resistance(g, qu, qv)
    assert float(np.max(np.abs(R - Ro) / Ro)) <= TOL


def test_spilled_plans_are_refused_where_scratch_is_fixed(P):
    """The batched sweep and the no-allocation entry point keep their scratch layouts fixed;
    they refuse a plan with fronts in global memory instead of running it."""
    import torch
    ctx = P.Context(0)
    g = I.grid2d(30, 31, seed=82)
    opt = P.Options()
    opt.front_smem = 1
    sym = P.Symbolic.of(g, options=opt)
    num = P.Numeric(ctx, sym)
    with pytest.raises(P.PeersError) as e:
        P.Batch(ctx, [sym], [num])
    assert e.value.status == P.EINVAL
    out = torch.empty(sym.nq, dtype=torch.float64, device="cuda:0")
    with pytest.raises(P.PeersError) as e:
        P.query_noalloc(ctx, sym, num, out)
    assert e.value.status == P.EINVAL
