"""peers_query_noalloc: the sweep for callers that cannot let the library allocate device
memory (a framework that owns all device memory through its own pool, or a latency-bound
loop that cannot afford the synchronisation an allocation may cause).  It must return what
peers_query returns, call after call, while its scratch lives in the library's static device
array.  This file is collected last so that a failure here leaves every other test already
run."""
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


def test_noalloc_matches_query_on_two_calls_in_a_row(P):
    import torch
    g = I.pdn3(side=21, seed=31)
    u, v = g.all_edges()
    pu, pv = I.random_pairs(g.n, 300, seed=32)           # two-branch pairs too
    qu = np.concatenate([u, pu, [7]]).astype(np.int32)
    qv = np.concatenate([v, pv, [7]]).astype(np.int32)   # and one u == v query
    opt = P.Options()
    opt.carry_budget = 8 << 20     # carry budget (bytes) inside the 16 MiB static scratch
    ctx = P.Context(0)
    sym = P.Symbolic.of(g, 0, qu, qv, True, opt)
    num = P.Numeric(ctx, sym)
    ref = P.query(ctx, sym, num)                          # the existing entry point
    nz = ref != 0
    assert np.count_nonzero(~nz) == 1
    for call in range(2):
        out = torch.full((sym.nq,), float("nan"), dtype=torch.float64, device="cuda:0")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(0)[0]
        P.query_noalloc(ctx, sym, num, out)
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the module that holds the static array
            assert torch.cuda.mem_get_info(0)[0] == free_before
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])) <= TOL
        assert np.all(got[~nz] == 0.0)


def test_noalloc_fits_any_plan_under_a_16_mib_budget(P):
    """A carry budget equal to the static buffer's 16 MiB must give a plan that fits it, here
    with several waves (more queries than one wave of the budget holds)."""
    import torch
    g = I.grid2d(200, 200, seed=34)
    opt = P.Options()
    opt.carry_budget = 16 << 20
    ctx = P.Context(0)
    sym = P.Symbolic.of(g, options=opt)
    info = sym.info()
    slot_bytes = 8 * (info["max_nb"] + 1)
    assert sym.nq > (16 << 20) // slot_bytes      # more than one wave
    num = P.Numeric(ctx, sym)
    ref = P.query(ctx, sym, num)
    for _ in range(2):
        out = torch.full((sym.nq,), float("nan"), dtype=torch.float64, device="cuda:0")
        P.query_noalloc(ctx, sym, num, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref) / np.abs(ref)) <= TOL


def test_noalloc_rejects_bad_result_buffers(P):
    """The binding refuses a result buffer the kernels could not write safely."""
    import torch
    g = I.grid2d(12, 13, seed=35)
    ctx = P.Context(0)
    sym = P.Symbolic.of(g)
    num = P.Numeric(ctx, sym)
    for bad in (np.empty(sym.nq),                                              # host array
                torch.empty(sym.nq, dtype=torch.float32, device="cuda:0"),     # float32
                torch.empty(sym.nq - 1, dtype=torch.float64, device="cuda:0"),  # too short
                torch.empty(2 * sym.nq, dtype=torch.float64, device="cuda:0")[::2]):  # strided
        with pytest.raises(ValueError):
            P.query_noalloc(ctx, sym, num, bad)


def test_noalloc_rejects_a_plan_larger_than_its_scratch(P):
    import torch
    g = I.grid2d(200, 200, seed=33)   # default plan: one wave of 79 600 queries
    ctx = P.Context(0)
    sym = P.Symbolic.of(g)
    num = P.Numeric(ctx, sym)
    out = torch.empty(sym.nq, dtype=torch.float64, device="cuda:0")
    with pytest.raises(P.PeersError) as e:
        P.query_noalloc(ctx, sym, num, out)
    assert e.value.status == P.EINVAL
    assert "static buffer" in str(e.value)
