"""Host-side tests of the C-ABI library (no GPU): the exported symbols, input validation and
the structure produced by peers_analyze."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2606_31535_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2606_31535_b300 import build, peers
    build.build()
    peers.load()
    return peers


def declared_functions():
    src = open(os.path.join(ROOT, "include", "peers.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(peers_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(P):
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(P.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name


def test_strerror_and_version(P):
    lib = P.load()
    assert lib.peers_strerror(0) == b"ok"
    assert lib.peers_strerror(P.ENOTSPD)
    assert b"sm_103a" in lib.peers_version()


def _bad(P, g, **kw):
    with pytest.raises(P.PeersError) as e:
        P.Symbolic(g.n, g.indptr, g.indices, g.w, **kw)
    return e.value.status


def test_rejects_malformed_graphs(P):
    g = I.grid2d(6, 7, seed=1)
    w = g.w.copy()
    w[3] = -1.0
    assert _bad(P, I.Graph(g.n, g.indptr, g.indices, w)) == P.EINVAL
    w = g.w.copy()
    w[5] = np.nan
    assert _bad(P, I.Graph(g.n, g.indptr, g.indices, w)) == P.EINVAL
    w = g.w.copy()
    w[0] *= 2.0   # (u,v) and (v,u) differ
    assert _bad(P, I.Graph(g.n, g.indptr, g.indices, w)) == P.EINVAL
    idx = g.indices.copy()
    idx[0] = 0    # self-loop at node 0
    assert _bad(P, I.Graph(g.n, g.indptr, idx, g.w)) == P.EINVAL
    assert _bad(P, g, ground=g.n) == P.EINVAL
    # two disjoint grids
    a = I.grid2d(4, 4, seed=2)
    u, v = a.all_edges()
    ww = a.edge_weights()
    two = I.from_edges(32, np.concatenate([u, u + 16]), np.concatenate([v, v + 16]),
                       np.concatenate([ww, ww]))
    assert _bad(P, two) == P.ENOTCONNECTED
    assert _bad(P, two, ground=20) == P.ENOTCONNECTED
    # a path 1-2-3-4 and an isolated node 0, grounded at the isolated node and on the path
    path = I.from_edges(5, np.array([1, 2, 3]), np.array([2, 3, 4]), np.ones(3))
    assert _bad(P, path, ground=0) == P.ENOTCONNECTED
    assert _bad(P, path, ground=2) == P.ENOTCONNECTED
    # connected once the ground's edges are counted: a star grounded at its centre
    star = I.from_edges(6, np.zeros(5, np.int64), np.arange(1, 6), np.ones(5))
    P.Symbolic(star.n, star.indptr, star.indices, star.w, ground=0).close()
    with pytest.raises(P.PeersError):
        P.Symbolic(g.n, g.indptr, g.indices, g.w, qu=np.array([0]), qv=np.array([g.n]))


def test_duplicate_edge_rejected(P):
    g = I.from_edges(3, np.array([0, 0, 1]), np.array([1, 1, 2]), np.array([1.0, 1.0, 1.0]))
    assert _bad(P, g) == P.EINVAL


@pytest.mark.parametrize("maker,use_coords", [
    (I.grid32, True), (I.grid32, False),
    (lambda: I.pdn3(side=33, seed=3), True),
    (lambda: I.rgg(4000, seed=4), True), (lambda: I.rgg(4000, seed=4), False),
    (lambda: I.grid_deleted(40, 45, seed=5), False),
])
def test_supernodal_structure(P, maker, use_coords):
    """Supernodes partition the columns, parents come later, levels are heights, and the
    elimination order is a permutation of the reduced nodes."""
    g = maker()
    sym = P.Symbolic.of(g, use_coords=use_coords)
    inf = sym.info()
    ex = sym.export()
    nr, ns = inf["n_reduced"], inf["nsuper"]
    assert nr == g.n - 1
    assert np.array_equal(np.sort(ex["perm"]), np.arange(nr))
    first = ex["first"]
    assert first[0] == 0 and first[-1] == nr and np.all(np.diff(first) > 0)
    par = ex["parent"]
    assert np.all((par == -1) | (par > np.arange(ns)))
    lev = ex["level"]
    for s in range(ns):
        if par[s] != -1:
            assert lev[par[s]] > lev[s]
    assert inf["levels"] == lev.max() + 1
    # roots have no rows below the diagonal; others do
    assert np.all((par == -1) == (ex["nb"] == 0))
    # the analysis counts at least as much executed work as walk work
    assert inf["walk_fma"] >= inf["walk_entries"] > 0
    assert inf["nnz_l"] >= inf["nnz_a"] + nr


def test_walk_work_matches_a_direct_count(P):
    """W from the analysis equals a count done here from the exported structure."""
    g = I.grid2d(12, 12, seed=6)
    sym = P.Symbolic.of(g)
    inf, ex = sym.info(), sym.export()
    first, par, nb = ex["first"], ex["parent"], ex["nb"]
    pos = np.empty(g.n - 1, np.int64)
    pos[ex["perm"]] = np.arange(g.n - 1)
    col2sn = np.repeat(np.arange(first.size - 1), np.diff(first))

    # rows of each supernode, rebuilt by brute force from the elimination of L_r's pattern
    n1 = g.n - 1
    A = np.zeros((n1, n1), bool)
    rows = np.repeat(np.arange(g.n), np.diff(g.indptr))
    for a, b in zip(rows, g.indices):
        if a and b:
            A[pos[a - 1], pos[b - 1]] = True
    Lp = A.copy()
    for k in range(n1):   # symbolic elimination
        nzr = np.flatnonzero(Lp[k + 1:, k]) + k + 1
        Lp[np.ix_(nzr, nzr)] = True
    # supernode's rows below its columns: union of its columns' patterns
    W = 0
    u, v = g.all_edges()
    for a, b in zip(u, v):
        pa, pb = (pos[x - 1] if x else -1 for x in (a, b))
        lo = max(pa, pb) if min(pa, pb) < 0 else min(pa, pb)
        s = col2sn[lo]
        fc = lo - first[s]
        while s != -1:
            nc = first[s + 1] - first[s]
            np_ = nc - fc
            W += np_ * (np_ - 1) // 2 + nb[s] * np_ + np_
            if par[s] == -1:
                break
            # first non-zero column in the parent: the parent-local row of the smallest row
            # below s
            below = np.flatnonzero(Lp[first[s + 1]:, first[s + 1] - 1]) + first[s + 1]
            fc = below[0] - first[par[s]]
            s = par[s]
    assert W == inf["walk_entries"]


def _lower_pattern(g, perm, ground):
    """Strictly-lower pattern of L (dense bool, n-1 x n-1) by symbolic elimination of the
    grounded graph in the order perm (perm[k] = reduced node eliminated k-th)."""
    n1 = g.n - 1
    pos = np.empty(n1, np.int64)
    pos[perm] = np.arange(n1)
    rows = np.repeat(np.arange(g.n), np.diff(g.indptr))
    L = np.zeros((n1, n1), bool)
    for a, b in zip(rows, g.indices):
        if a != ground and b != ground:
            i, j = pos[a - (a > ground)], pos[b - (b > ground)]
            if i > j:
                L[i, j] = True
    for k in range(n1):   # eliminating k joins all of its lower neighbours
        nz = np.flatnonzero(L[k + 1:, k]) + k + 1
        if nz.size > 1:
            L[np.ix_(nz, nz)] |= np.tril(np.ones((nz.size, nz.size), bool), -1)
    return L


def _small_graphs():
    rng = np.random.default_rng(21)
    out = []
    n = 120   # random tree
    out.append(("tree", I.from_edges(n, np.arange(1, n), rng.integers(0, np.arange(1, n)),
                                     rng.uniform(0.5, 2.0, n - 1)), 7))
    n = 40    # star grounded at its centre: the reduced graph has no edges
    out.append(("star-centre", I.from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n),
                                            np.ones(n - 1)), 0))
    out.append(("star-leaf", I.from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n),
                                          np.ones(n - 1)), 5))
    iu, iv = np.triu_indices(14, 1)   # complete graph
    out.append(("K14", I.from_edges(14, iu, iv, np.ones(iu.size)), 3))
    n = 200   # path with random chords
    cu, cv = rng.integers(0, n, 60), rng.integers(0, n, 60)
    eu, ev = np.concatenate([np.arange(n - 1), cu]), np.concatenate([np.arange(1, n), cv])
    keep = eu != ev
    a, b = np.minimum(eu, ev)[keep], np.maximum(eu, ev)[keep]
    key = np.unique(a * n + b)
    out.append(("chords", I.from_edges(n, key // n, key % n, np.ones(key.size)), 123))
    out.append(("grid", I.grid2d(11, 13, seed=4), 60))
    out.append(("rgg", I.rgg(250, seed=8), 17))
    return out


@pytest.mark.parametrize("name,g,ground", [pytest.param(*c, id=c[0]) for c in _small_graphs()])
def test_supernode_rows_match_symbolic_elimination(P, name, g, ground):
    """Each supernode's below-diagonal row count equals the column count of its last column in
    L's pattern, found here by eliminating the grounded graph in the exported order; every
    column of the supernode has its lower rows within that set; the parent holds the
    smallest of those rows."""
    for use_coords in ((True, False) if g.coords is not None else (False,)):
        sym = P.Symbolic.of(g, ground=ground, use_coords=use_coords)
        ex = sym.export()
        first, par, nb = ex["first"], ex["parent"], ex["nb"]
        L = _lower_pattern(g, ex["perm"], ground)
        col2sn = np.repeat(np.arange(first.size - 1), np.diff(first))
        for f in range(first.size - 1):
            last = first[f + 1] - 1
            below = np.flatnonzero(L[last + 1:, last]) + last + 1
            assert nb[f] == below.size, (name, f)
            for k in range(first[f], last):
                rows_k = np.flatnonzero(L[last + 1:, k]) + last + 1
                assert np.isin(rows_k, below).all(), (name, f, k)
            assert par[f] == (col2sn[below[0]] if below.size else -1), (name, f)


def test_all_edge_order_and_footprint(P):
    g = I.grid32()
    sym = P.Symbolic.of(g)
    assert sym.nq == g.m
    assert sym.footprint_bytes() > 8 * sym.info()["nnz_l"]


def test_two_branch_pairs_are_planned(P):
    g = I.grid2d(30, 30, seed=1)
    u, v = I.random_pairs(g.n, 500, seed=3)
    inf = P.Symbolic.of(g, qu=u, qv=v).info()
    assert inf["nq"] == 500
    assert 0 < inf["nq_two_branch"] <= 500
    assert inf["walk_fma"] >= inf["walk_entries"] > 0


def test_analysis_does_not_depend_on_host_threads(P, monkeypatch):
    """One host thread and eight give the same ordering, supernodes and plan.

    A 1025 x 1024 grid (1 049 600 nodes, 4.2M stored entries, 2.1M all-edge queries) is large
    enough for every threaded step: validation chunks, nested-dissection splits of 2^20 nodes
    or more, per-thread query chunks and per-level plan items.
    """
    g = I.grid2d(1025, 1024, seed=12)
    assert g.n - 1 >= 1 << 20
    many_waves = P.Options()
    many_waves.carry_budget = 1 << 30   # a few tens of waves
    for opt in (None, many_waves):
        runs = []
        for threads in ("1", "8"):
            monkeypatch.setenv("PEERS_ANALYSIS_THREADS", threads)
            sym = P.Symbolic.of(g, options=opt)
            inf = {k: v for k, v in sym.info().items() if not k.startswith("t_")}
            inf["footprint"] = sym.footprint_bytes()
            runs.append((inf, sym.export()))
            sym.close()
        assert runs[0][0] == runs[1][0]
        for key in runs[0][1]:
            assert np.array_equal(runs[0][1][key], runs[1][1][key]), key
        if opt is None:
            one_wave = runs[0][0]
    # the waves (a smaller carry buffer) split the same walk
    assert runs[0][0]["footprint"] < one_wave["footprint"] - (1 << 30)
    assert runs[0][0]["walk_entries"] == one_wave["walk_entries"]


def test_wave_budget_option(P):
    g = I.grid2d(20, 20, seed=2)
    opt = P.Options()
    opt.carry_budget = 64 * 1024
    small = P.Symbolic.of(g, options=opt)
    big = P.Symbolic.of(g)
    assert small.footprint_bytes() < big.footprint_bytes()
    assert small.info()["walk_entries"] == big.info()["walk_entries"]


def test_route_plan_costs_concurrent_and_cached(P):
    """The block-inverse and selected-inversion plans are built once per symbolic handle and
    shared; cost queries from several host threads at once (ctypes releases the GIL) must all
    see the same numbers as a fresh handle, built or cached."""
    import threading
    g = I.pdn3(side=65, seed=91)
    lib = P.load()
    a, b = P.Symbolic.of(g), P.Symbolic.of(g)   # keep the handles alive across the calls
    fresh = [(lib.peers_blockinv_fma(a._h), lib.peers_selinv_fma(b._h))]
    sym = P.Symbolic.of(g)
    out, errs = [], []

    def worker():
        try:
            for _ in range(3):
                out.append((lib.peers_blockinv_fma(sym._h), lib.peers_selinv_fma(sym._h),
                            lib.peers_blockinv_bytes(sym._h)))
        except Exception as e:   # pragma: no cover - reported below
            errs.append(e)

    threads = [threading.Thread(target=worker) for _ in range(6)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errs
    assert len(out) == 18
    assert all(o[:2] == fresh[0] for o in out)
    assert len({o[2] for o in out}) == 1 and out[0][2] > 0
    assert fresh[0][0] > 0 and fresh[0][1] > 0


def test_small_front_budget_moves_fronts_to_global_memory(P):
    """A lowered shared-memory budget marks the supernodes whose fronts no longer fit (their
    sweep fronts go to global memory) without changing the work of any query."""
    g = I.grid2d(60, 61, seed=91)
    base = P.Symbolic.of(g).info()
    assert base["nsuper_spilled"] == 0
    counts = []
    for fs in (1, 4 << 10, 64 << 10):
        opt = P.Options()
        opt.front_smem = fs
        info = P.Symbolic.of(g, options=opt).info()
        assert info["walk_entries"] == base["walk_entries"]
        counts.append(info["nsuper_spilled"])
    assert counts[0] == base["nsuper"] and 0 < counts[1] < base["nsuper"] and counts[2] == 0


def test_one_stream_option_removes_lanes_and_split_blocks(P):
    """The default plan of a mesh with wide separators spreads independent subtrees over the
    lanes and splits the factorization's multi-block updates; peers_options.one_stream keeps
    the same supernodes and work on one stream."""
    g = I.grid2d(200, 200, seed=11, law="loguniform", lo=1e-3, hi=1e3)
    base = P.Symbolic.of(g).info()
    assert base["lanes"] == 4 and base["split_blocks"] > 0
    opt = P.Options()
    opt.one_stream = 1
    info = P.Symbolic.of(g, options=opt).info()
    assert info["lanes"] == 0 and info["split_blocks"] == 0
    for k in ("nsuper", "levels", "nnz_l", "walk_entries", "factor_fma"):
        assert info[k] == base[k]


def _walk_entries_by_solve(g, ex, ground, qu, qv):
    """W of a query list, counted here from the pattern of the sparse solve L y = e_lo - e_hi
    (§III-G, eq. 16-18): y is non-zero on the etree paths from both endpoints to the root, so a
    supernode is visited from the first of its columns that either path reaches; the visit
    reads the panel entries from that column on (its triangle, its n_b rows below and the
    diagonal).  Supernode parents and the columns where the paths enter them come from the
    symbolic elimination of the grounded graph in the exported order."""
    first, par, nb = ex["first"], ex["parent"], ex["nb"]
    L = _lower_pattern(g, ex["perm"], ground)
    n1 = g.n - 1
    pos = np.empty(n1, np.int64)
    pos[ex["perm"]] = np.arange(n1)
    col2sn = np.repeat(np.arange(first.size - 1), np.diff(first))
    enter = []   # per supernode, the column where a path from below enters its parent
    for s in range(first.size - 1):
        last = first[s + 1] - 1
        below = np.flatnonzero(L[last + 1:, last]) + last + 1
        enter.append(int(below[0]) if below.size else -1)
    W = 0
    for a, b in zip(qu, qv):
        if a == b:
            continue
        reached = {}   # supernode -> first local column reached
        for x in (a, b):
            if x == ground:
                continue
            c = int(pos[x - (x > ground)])
            s = int(col2sn[c])
            while s != -1:
                loc = c - int(first[s])
                if s in reached:   # the rest of this path is already on the other one
                    reached[s] = min(reached[s], loc)
                    break
                reached[s] = loc
                c, s = enter[s], int(par[s])
        for s, fc in reached.items():
            m = int(first[s + 1] - first[s]) - fc
            W += m * (m - 1) // 2 + int(nb[s]) * m + m
    return W


@pytest.mark.parametrize("name,g,ground", [pytest.param(*c, id=c[0]) for c in _small_graphs()])
def test_walk_work_of_listed_pairs_matches_the_solve_pattern(P, name, g, ground):
    """The analysis's W (the walk's entries, the roofline's algorithmic work) for a query list
    mixing edges, non-adjacent pairs (one- and two-branch walks), pairs through the ground and
    u == v equals the count from the solve's pattern, with and without coordinates and with a
    small carry budget (many waves)."""
    rng = np.random.default_rng(len(name) * 7 + ground)
    k = 300
    qu = rng.integers(0, g.n, k).astype(np.int32)
    qv = rng.integers(0, g.n, k).astype(np.int32)
    eu, ev = g.all_edges()
    pick = rng.integers(0, eu.size, 60) if eu.size else np.zeros(0, np.int64)
    qu = np.concatenate([qu, eu[pick], [ground, ground, 3 % g.n]]).astype(np.int32)
    qv = np.concatenate([qv, ev[pick], [(ground + 1) % g.n, ground, 3 % g.n]]).astype(np.int32)
    few = P.Options()
    few.carry_budget = 4096
    for use_coords in ((True, False) if g.coords is not None else (False,)):
        for opt in (None, few):
            sym = P.Symbolic.of(g, ground=ground, qu=qu, qv=qv, use_coords=use_coords,
                                options=opt)
            inf, ex = sym.info(), sym.export()
            assert inf["walk_entries"] == _walk_entries_by_solve(g, ex, ground, qu, qv), \
                (name, use_coords, opt is not None)
            sym.close()


def test_binding_checks_buffer_sizes_before_the_library_reads_them(P):
    """The library reads n + 1 offsets, indptr[n] indices and conductances, nq query pairs,
    n x dim coordinates and (for a refactor) one conductance per stored entry through plain
    pointers; the binding rejects arrays of other sizes before the call, and the
    sparsifier's inputs unless they are float64 CUDA tensors (checked before any device
    work, so this runs without a GPU)."""
    import torch
    g = I.grid2d(5, 6, seed=3)
    with pytest.raises(ValueError):
        P.Symbolic(g.n, g.indptr[:-1], g.indices, g.w)
    with pytest.raises(ValueError):
        P.Symbolic(g.n, g.indptr, g.indices[:-2], g.w[:-2])
    with pytest.raises(ValueError):
        P.Symbolic(g.n, g.indptr, g.indices, g.w[:-1])
    with pytest.raises(ValueError):
        P.Symbolic(g.n, g.indptr, g.indices, g.w, qu=np.array([0, 1]), qv=np.array([2]))
    with pytest.raises(ValueError):
        P.Symbolic(g.n, g.indptr, g.indices, g.w, coords=g.coords[:-1])
    sym = P.Symbolic.of(g)
    assert sym.nnz == g.indices.size
    with pytest.raises(ValueError):
        P.Numeric(None, sym, g.w[:-1])
    sym.close()
    w = torch.ones(4, dtype=torch.float64)
    with pytest.raises(ValueError):   # host tensors
        P.sparsify(None, w, w, w)
    with pytest.raises(ValueError):
        P.sparsify(None, np.ones(4), np.ones(4), np.ones(4))
