"""The factorization's, the selected inversion's and the block inverse's concurrent
schedules against the one-stream schedule (peers_options.one_stream).  The lanes run independent subtrees on
their own streams. A factorization column block of more than one block runs its update
split over three streams: the next block's columns on a high-priority chain, the panel's
other columns, and the update matrix. Every entry still takes its updates in the same
order, so every route's results are equal bit for bit.
"""
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


def graph(name):
    if name == "grid-200":
        return I.grid2d(200, 200, seed=11, law="loguniform", lo=1e-3, hi=1e3)
    return I.pdn3(side=81, seed=8)


def routes(P, ctx, g, one_stream):
    import torch
    opt = P.Options()
    opt.one_stream = one_stream
    sym = P.Symbolic.of(g, options=opt)
    num = P.Numeric(ctx, sym)
    out = {}
    out["walk"] = P.query(ctx, sym, num)
    for name, fn in (("selinv", P.query_selinv), ("blockinv", P.query_blockinv)):
        R = torch.empty(sym.nq, dtype=torch.float64, device="cuda:0")
        fn(ctx, sym, num, R)
        out[name] = R.cpu().numpy()
    return out, sym.info()


@pytest.mark.parametrize("name", ["grid-200", "pdn3-81"])
def test_concurrent_schedules_match_one_stream_bit_for_bit(P, name):
    ctx = P.Context(0)
    g = graph(name)
    ref, info1 = routes(P, ctx, g, 1)
    got, info = routes(P, ctx, g, 0)
    assert info1["lanes"] == 0 and info1["split_blocks"] == 0
    assert info["lanes"] > 0 and info["split_blocks"] > 0
    for k in ("walk", "selinv", "blockinv"):
        a, b = np.asarray(got[k]), np.asarray(ref[k])
        assert a.shape == b.shape and np.array_equal(a.view(np.int64), b.view(np.int64)), k
