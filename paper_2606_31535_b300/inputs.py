"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and bench.py.

This module only builds graphs and query lists (topology, conductances, coordinates).  It
holds none of the effective-resistance arithmetic, so both sides of a parity test can use
it without sharing any part of the method.

The workloads stand in for the resistive networks the paper evaluates (§V-A: IBM power
grids, SuiteSparse circuit/thermal matrices, industrial macros), which are not available
here.  Every generator draws from ``numpy.random.Generator(PCG64(seed))``.

Conventions (the paper's problem statement, §II-A, eq. 1):
  * a graph is an undirected weighted graph G=(V,E,w) with positive conductances;
  * it is returned as a symmetric CSR (``indptr`` int64, ``indices`` int32 sorted within
    each row, ``w`` float64 per stored entry), no self-loops, no duplicate edges;
  * "all edges" means, for u ascending, every CSR neighbour v > u in CSR order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Graph:
    n: int
    indptr: np.ndarray      # int64 [n+1]
    indices: np.ndarray     # int32 [nnz]
    w: np.ndarray           # float64 [nnz]
    coords: np.ndarray | None = None   # float64 [n, dim] (layout hint only)
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.indices.size // 2)

    def all_edges(self) -> tuple[np.ndarray, np.ndarray]:
        """Edge list (u < v) in the all-edge order: u ascending, then CSR order."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.indptr))
        keep = self.indices > rows
        return rows[keep].astype(np.int32), self.indices[keep].astype(np.int32)

    def edge_weights(self) -> np.ndarray:
        """Conductance of every edge in :meth:`all_edges` order."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.indptr))
        keep = self.indices > rows
        return self.w[keep].copy()


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _draw(rng: np.random.Generator, k: int, law: str, lo: float, hi: float) -> np.ndarray:
    if law == "uniform":
        return rng.uniform(lo, hi, size=k)
    if law == "loguniform":
        return 10.0 ** rng.uniform(math.log10(lo), math.log10(hi), size=k)
    raise ValueError(f"unknown conductance law {law!r}")


def from_edges(n: int, eu: np.ndarray, ev: np.ndarray, ew: np.ndarray,
               coords: np.ndarray | None = None, name: str = "") -> Graph:
    """Symmetric CSR (indices sorted within each row) from an undirected edge list."""
    eu = np.asarray(eu, dtype=np.int64)
    ev = np.asarray(ev, dtype=np.int64)
    ew = np.asarray(ew, dtype=np.float64)
    src = np.concatenate([eu, ev])
    dst = np.concatenate([ev, eu])
    wt = np.concatenate([ew, ew])
    order = np.lexsort((dst, src))
    src, dst, wt = src[order], dst[order], wt[order]
    counts = np.bincount(src, minlength=n)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    return Graph(n, indptr, dst.astype(np.int32), wt, coords, name)


def _grid_edges(rows: int, cols: int, base: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Edges of a rows x cols 5-point grid in draw order: row-major nodes, for each node
    its right edge then its down edge."""
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    node = (r * cols + c).ravel() + base
    right_ok = (c < cols - 1).ravel()
    down_ok = (r < rows - 1).ravel()
    # interleave (right, down) per node, dropping the missing ones
    u = np.stack([node, node], axis=1).ravel()
    v = np.stack([node + 1, node + cols], axis=1).ravel()
    ok = np.stack([right_ok, down_ok], axis=1).ravel()
    return u[ok], v[ok]


def grid2d(rows: int, cols: int, seed: int, law: str = "uniform",
           lo: float = 0.5, hi: float = 2.0) -> Graph:
    """2-D 5-point grid; node id r*cols+c; coordinates (c, r)."""
    rng = _rng(seed)
    eu, ev = _grid_edges(rows, cols)
    ew = _draw(rng, eu.size, law, lo, hi)
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    coords = np.stack([c.ravel(), r.ravel()], axis=1).astype(np.float64)
    return from_edges(rows * cols, eu, ev, ew, coords, f"grid{rows}x{cols}")


def pdn3(side: int = 577, layers: int = 3, via_stride: int = 4, seed: int = 2,
         lo: float = 1e-2, hi: float = 1e2) -> Graph:
    """Power-delivery-network-like mesh: ``layers`` stacked side x side 5-point grids, with
    a via between consecutive layers at every node whose row and column are multiples of
    ``via_stride``.  Conductances log-uniform in [lo, hi].  Draw order: layer by layer
    (row-major, right edge then down edge), then the vias layer pair by layer pair in
    row-major order.  Node id = layer*side^2 + r*side + c; coordinates (c, r, layer)."""
    rng = _rng(seed)
    per = side * side
    us, vs = [], []
    for layer in range(layers):
        u, v = _grid_edges(side, side, base=layer * per)
        us.append(u)
        vs.append(v)
    rr, cc = np.meshgrid(np.arange(0, side, via_stride), np.arange(0, side, via_stride),
                         indexing="ij")
    via_local = (rr * side + cc).ravel()
    for layer in range(layers - 1):
        us.append(via_local + layer * per)
        vs.append(via_local + (layer + 1) * per)
    eu = np.concatenate(us)
    ev = np.concatenate(vs)
    ew = _draw(rng, eu.size, "loguniform", lo, hi)
    L, r, c = np.meshgrid(np.arange(layers), np.arange(side), np.arange(side), indexing="ij")
    coords = np.stack([c.ravel(), r.ravel(), L.ravel()], axis=1).astype(np.float64)
    return from_edges(layers * per, eu, ev, ew, coords, f"pdn{layers}x{side}x{side}")


def grid_deleted(rows: int, cols: int, seed: int, frac: float = 0.05,
                 lo: float = 1e-2, hi: float = 1e2) -> Graph:
    """Grid with ``frac`` of its edges deleted while keeping it connected: a random spanning
    tree (Kruskal on seeded random keys) is kept and round(frac*m) edges are deleted
    uniformly among the non-tree edges.  Conductances log-uniform, drawn for the surviving
    edges in grid draw order."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree

    rng = _rng(seed)
    eu, ev = _grid_edges(rows, cols)
    m = eu.size
    keys = rng.random(m)
    # Kruskal on the seeded keys = the minimum spanning tree for those (distinct) keys
    n = rows * cols
    mst = minimum_spanning_tree(coo_matrix((keys + 1.0, (eu, ev)), shape=(n, n))).tocoo()
    in_tree = set(zip(np.minimum(mst.row, mst.col).tolist(), np.maximum(mst.row, mst.col).tolist()))
    tree = np.fromiter(((int(a), int(b)) in in_tree for a, b in zip(eu, ev)), dtype=bool, count=m)
    non_tree = np.flatnonzero(~tree)
    k = int(round(frac * m))
    drop = rng.choice(non_tree, size=min(k, non_tree.size), replace=False)
    keep = np.ones(m, dtype=bool)
    keep[drop] = False
    eu, ev = eu[keep], ev[keep]
    ew = _draw(rng, eu.size, "loguniform", lo, hi)
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    coords = np.stack([c.ravel(), r.ravel()], axis=1).astype(np.float64)
    return from_edges(rows * cols, eu, ev, ew, coords, f"gridx{rows}x{cols}")


def rgg(n: int, seed: int, mean_degree: float = 6.0, lo: float = 1e-2, hi: float = 1e2) -> Graph:
    """Random geometric graph: n uniform points in the unit square, radius
    sqrt(mean_degree/(pi*n)), no wrap.  Each component other than the largest is joined to
    the largest by one edge from its first node to that node's nearest neighbour in the
    largest component.  Conductances log-uniform, drawn after the topology (pairs in
    lexicographic order, then the joining edges)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    from scipy.spatial import cKDTree

    rng = _rng(seed)
    pts = rng.random((n, 2))
    radius = math.sqrt(mean_degree / (math.pi * n))
    tree = cKDTree(pts)
    pairs = tree.query_pairs(radius, output_type="ndarray")
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    eu, ev = pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)
    a = coo_matrix((np.ones(eu.size), (eu, ev)), shape=(n, n))
    ncomp, label = connected_components(a, directed=False)
    if ncomp > 1:
        sizes = np.bincount(label)
        giant = int(np.argmax(sizes))
        gidx = np.flatnonzero(label == giant)
        gtree = cKDTree(pts[gidx])
        extra_u, extra_v = [], []
        for comp in range(ncomp):
            if comp == giant:
                continue
            first = int(np.flatnonzero(label == comp)[0])
            _, j = gtree.query(pts[first])
            extra_u.append(min(first, int(gidx[j])))
            extra_v.append(max(first, int(gidx[j])))
        eu = np.concatenate([eu, np.asarray(extra_u, dtype=np.int64)])
        ev = np.concatenate([ev, np.asarray(extra_v, dtype=np.int64)])
    ew = _draw(rng, eu.size, "loguniform", lo, hi)
    return from_edges(n, eu, ev, ew, pts.astype(np.float64), f"rgg{n}")


# ---------------------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------------------

def grid32() -> Graph:
    """32x32 5-point grid, conductances uniform in [0.5, 2], seed 1 (1024 nodes, 1984 edges)."""
    return grid2d(32, 32, seed=1, law="uniform", lo=0.5, hi=2.0)


def pdn1m() -> Graph:
    """3-layer 577x577 PDN mesh, vias every 4th node, log-uniform 1e-2..1e2, seed 2
    (998 787 nodes, 2 036 162 edges)."""
    return pdn3(577, 3, 4, seed=2)


def grid4096() -> Graph:
    """4096x4096 5-point grid, log-uniform 1e-3..1e3, seed 5 (16.7M nodes, 33.5M edges)."""
    return grid2d(4096, 4096, seed=5, law="loguniform", lo=1e-3, hi=1e3)


def batch_graphs(count: int = 256, base_seed: int = 3000) -> list[Graph]:
    """Many independent connected graphs of uneven size: n_i = round(exp U(ln 1024,
    ln 65536)) drawn from seed base_seed+i; even i are near-square grids with 5% of edges
    deleted, odd i are random geometric graphs of mean degree 6."""
    out = []
    for i in range(count):
        rng = _rng(base_seed + i)
        ni = int(round(math.exp(rng.uniform(math.log(1024), math.log(65536)))))
        if i % 2 == 0:
            r = int(round(math.sqrt(ni)))
            c = int(round(ni / r))
            out.append(grid_deleted(r, c, seed=base_seed + i))
        else:
            out.append(rgg(ni, seed=base_seed + i))
    return out


def query_subset(g: Graph, frac: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Seeded uniform subset of the edges (kept in all-edge order)."""
    u, v = g.all_edges()
    rng = _rng(seed)
    k = max(1, int(round(frac * u.size)))
    pick = np.sort(rng.choice(u.size, size=k, replace=False))
    return u[pick], v[pick]


def random_pairs(n: int, k: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """k seeded node pairs (u != v), generally not edges."""
    rng = _rng(seed)
    u = rng.integers(0, n, size=k)
    v = rng.integers(0, n - 1, size=k)
    v = v + (v >= u)
    return u.astype(np.int32), v.astype(np.int32)


def serve_request(i: int, base_seed: int = 4, n_lo: int = 10_000, n_hi: int = 500_000):
    """Request i of the serving stream: n log-uniform in [n_lo, n_hi]; a near-square grid with
    5% of its edges deleted or a random geometric graph (mean degree 6), 50/50; all edges or a
    seeded uniform 10% subset of them, 50/50.  Returns (graph, qu, qv) with qu = qv = None for
    all edges."""
    rng = np.random.Generator(np.random.PCG64([base_seed, i]))
    n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    sub = int(rng.integers(0, 2 ** 31))
    if rng.random() < 0.5:
        r = int(round(math.sqrt(n)))
        g = grid_deleted(r, max(2, int(round(n / r))), seed=sub)
    else:
        g = rgg(n, seed=sub)
    if rng.random() < 0.5:
        return g, None, None
    qu, qv = query_subset(g, 0.1, seed=sub + 1)
    return g, qu, qv


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    rng = _rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
