"""Serving loop with continuous batching: every request's result equals its own single sweep
bit for bit (alone and in the mix), under memory-budget queueing, one-at-a-time admission and
failing requests."""
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


def requests():
    out = []
    for i in range(12):
        if i % 3 == 0:
            g = I.grid_deleted(30 + 9 * i, 33 + 7 * i, seed=200 + i)
        elif i % 3 == 1:
            g = I.rgg(1500 + 700 * i, seed=200 + i)
        else:
            g = I.pdn3(side=17 + 2 * i, seed=200 + i)
        if i % 4 == 1:
            qu, qv = I.query_subset(g, 0.1, seed=300 + i)
        elif i % 4 == 2:
            qu, qv = I.random_pairs(g.n, 500, seed=300 + i)
        else:
            qu = qv = None
        out.append((g, qu, qv))
    return out


def alone(P, ctx, g, qu, qv):
    sym = P.Symbolic.of(g, 0, qu, qv)
    return P.query(ctx, sym, P.Numeric(ctx, sym)), sym.footprint_bytes()


@pytest.mark.parametrize("budget_mode,max_active", [("ample", 0), ("tight", 0), ("ample", 1)])
def test_served_results_equal_alone(P, oracle_mod, budget_mode, max_active):
    reqs = requests()
    ctx = P.Context(0)
    ref, feet = zip(*[alone(P, ctx, *r) for r in reqs])
    budget = 0 if budget_mode == "ample" else int(max(feet) * 1.05)
    sv = P.Server(0, mem_budget_bytes=budget, max_active=max_active, workers=3)
    tickets = [sv.submit(g, qu, qv) for g, qu, qv in reqs]
    for i, t in enumerate(tickets):
        R, lat = sv.wait(t)
        assert lat > 0
        assert np.array_equal(R, ref[i]), i
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["queries"] == sum(len(r) for r in ref)
    assert 0 < st["p50_s"] <= st["p99_s"]
    if budget_mode == "tight":
        assert st["peak_bytes"] <= budget
    sv.close()
    g, qu, qv = reqs[2]
    assert np.max(np.abs(ref[2] - oracle_mod.resistance(g, qu, qv)) / ref[2]) <= TOL


def test_failing_request_does_not_stop_the_server(P):
    a = I.grid2d(4, 4, seed=2)
    u, v = a.all_edges()
    ww = a.edge_weights()
    broken = I.from_edges(32, np.concatenate([u, u + 16]), np.concatenate([v, v + 16]),
                          np.concatenate([ww, ww]))   # two components
    good = I.grid2d(20, 21, seed=3)
    sv = P.Server(0, workers=2)
    tb = sv.submit(broken)
    tg = sv.submit(good)
    with pytest.raises(P.PeersError) as e:
        sv.wait(tb)
    assert e.value.status == P.ENOTCONNECTED
    R, _ = sv.wait(tg)
    ctx = P.Context(0)
    assert np.array_equal(R, alone(P, ctx, good, None, None)[0])
    st = sv.stats()
    assert st["completed"] == 1 and st["failed"] == 1
    sv.close()


def test_server_analysis_options_keep_results(P):
    """Options given to the server (here small tile caps and a small carry budget, which split
    the queries into more items and waves) apply to every request's analysis; column blocks
    stay aligned, so each result is still bit-identical to the default single sweep."""
    reqs = requests()[:6]
    ctx = P.Context(0)
    ref = [alone(P, ctx, *r)[0] for r in reqs]
    opt = P.Options()
    opt.qcap[:] = [4, 8, 2, 16]
    opt.carry_budget = 8 << 20
    sv = P.Server(0, workers=2, options=opt)
    tickets = [sv.submit(g, qu, qv) for g, qu, qv in reqs]
    for i, t in enumerate(tickets):
        R, _ = sv.wait(t)
        assert np.array_equal(R, ref[i]), i
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    sv.close()


def test_requests_share_steps(P):
    """Continuous batching proper: requests held until all are factored, then released
    together, are swept in shared launches (a step carries work of several requests, and the
    steps run are fewer than the requests' own step counts added up), and every result is
    still bit-identical to its solo sweep."""
    import time
    reqs = requests()
    ctx = P.Context(0)
    ref = [alone(P, ctx, *r)[0] for r in reqs]
    sv = P.Server(0, workers=3)
    sv.hold(True)
    tickets = [sv.submit(g, qu, qv) for g, qu, qv in reqs]
    t0 = time.time()
    while sv.stats()["ready"] < len(reqs):
        assert time.time() - t0 < 120, "requests were not factored in time"
        time.sleep(0.01)
    sv.hold(False)
    for i, t in enumerate(tickets):
        R, _ = sv.wait(t)
        assert np.array_equal(R, ref[i]), i
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["max_step_requests"] >= 2
    assert st["steps"] < st["request_steps"]
    sv.close()
