"""CPU oracle for exact effective resistance -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The library's compute path never does, and the two share no code.

Two independent implementations of the paper's definition (PEERS §II-A eq. 2-4, §IV-A
eq. 15-18):

* :class:`Factor` / :func:`resistance` -- ``oracle.c``: own ordering, simplicial up-looking
  LDL^T, and per query a sparse forward solve over the union of the two etree paths (the
  paper's own error reference, LSolve, Alg. 2), R = sum_k y_k^2/d_k.
* :func:`dense_resistance` -- the textbook formula on the Laplacian's Moore-Penrose
  pseudo-inverse, R_uv = L+_uu + L+_vv - 2 L+_uv (the definition the paper starts from in §I),
  for small graphs.  It pins the sparse oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ERRORS = {-1: "invalid input", -2: "out of memory", -3: "matrix not positive definite"}


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into liboracle.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        lib.oracle_factorize.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_int, P(ctypes.c_void_p)]
        lib.oracle_factorize.restype = ctypes.c_int
        lib.oracle_resistance.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        lib.oracle_resistance.restype = ctypes.c_int
        lib.oracle_full_solve.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                          P(ctypes.c_double), P(ctypes.c_double)]
        lib.oracle_full_solve.restype = ctypes.c_int
        lib.oracle_nnz_l.argtypes = [ctypes.c_void_p]
        lib.oracle_nnz_l.restype = ctypes.c_int64
        lib.oracle_n.argtypes = [ctypes.c_void_p]
        lib.oracle_n.restype = ctypes.c_int64
        lib.oracle_export.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
        lib.oracle_export.restype = None
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        lib.oracle_free.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Factor:
    """Grounded, ordered and factored reduced Laplacian of one graph (oracle.c)."""

    def __init__(self, n, indptr, indices, w, ground=0, coords=None):
        lib = _load()
        self._keep = [np.ascontiguousarray(indptr, dtype=np.int64),
                      np.ascontiguousarray(indices, dtype=np.int32),
                      np.ascontiguousarray(w, dtype=np.float64)]
        c = None if coords is None else np.ascontiguousarray(coords, dtype=np.float64)
        dim = 0 if c is None else (c.shape[1] if c.ndim == 2 else 1)
        h = ctypes.c_void_p()
        st = lib.oracle_factorize(int(n), _ptr(self._keep[0]), _ptr(self._keep[1]),
                                  _ptr(self._keep[2]), int(ground), _ptr(c), dim, ctypes.byref(h))
        if st != 0:
            raise RuntimeError(f"oracle_factorize: {ERRORS.get(st, st)}")
        self._h = h
        self.n_graph = int(n)
        self.ground = int(ground)

    @classmethod
    def of(cls, g, ground=0, use_coords=True):
        return cls(g.n, g.indptr, g.indices, g.w, ground, g.coords if use_coords else None)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _load().oracle_free(h)
            self._h = None

    @property
    def nnz_l(self) -> int:
        return int(_load().oracle_nnz_l(self._h))

    def resistance(self, qu, qv, threads: int | None = None) -> np.ndarray:
        qu = np.ascontiguousarray(qu, dtype=np.int32)
        qv = np.ascontiguousarray(qv, dtype=np.int32)
        R = np.empty(qu.size, dtype=np.float64)
        if threads is None:
            threads = os.cpu_count() or 1
        st = _load().oracle_resistance(self._h, qu.size, _ptr(qu), _ptr(qv), int(threads), _ptr(R))
        if st != 0:
            raise RuntimeError(f"oracle_resistance: {ERRORS.get(st, st)}")
        return R

    def full_solve(self, u: int, v: int) -> tuple[float, float]:
        """(R, ||L_r x - b||_inf) by a complete forward/backward solve."""
        r, res = ctypes.c_double(), ctypes.c_double()
        st = _load().oracle_full_solve(self._h, int(u), int(v), ctypes.byref(r), ctypes.byref(res))
        if st != 0:
            raise RuntimeError(f"oracle_full_solve: {ERRORS.get(st, st)}")
        return r.value, res.value

    def export(self):
        """(d, etree parent, perm) in elimination order."""
        n = int(_load().oracle_n(self._h))
        d = np.empty(n, dtype=np.float64)
        par = np.empty(n, dtype=np.int32)
        perm = np.empty(n, dtype=np.int32)
        _load().oracle_export(self._h, _ptr(d), _ptr(par), _ptr(perm))
        return d, par, perm


def resistance(g, qu, qv, ground=0, threads=None, use_coords=True) -> np.ndarray:
    return Factor.of(g, ground, use_coords).resistance(qu, qv, threads)


def laplacian_dense(g) -> np.ndarray:
    """Dense combinatorial Laplacian L_G = D - W (eq. 1)."""
    L = np.zeros((g.n, g.n))
    rows = np.repeat(np.arange(g.n), np.diff(g.indptr))
    L[rows, g.indices] = -g.w
    L[np.arange(g.n), np.arange(g.n)] = -L.sum(axis=1)
    return L


def dense_resistance(g, qu, qv) -> np.ndarray:
    """R_uv = L+_uu + L+_vv - 2 L+_uv with L+ the pseudo-inverse of the Laplacian (numpy)."""
    Lp = np.linalg.pinv(laplacian_dense(g), hermitian=True)
    qu = np.asarray(qu, dtype=np.int64)
    qv = np.asarray(qv, dtype=np.int64)
    return Lp[qu, qu] + Lp[qv, qv] - 2.0 * Lp[qu, qv]


def sparsify(w, R, q, u):
    """Spectral sparsification by effective resistances, the paper's Alg. 1: q draws of an edge
    with probability p_e proportional to w_e R_e; each draw adds w_e / (q p_e) to its edge.
    The probabilities are the quantised ones the library documents (integer weights
    k_e = floor(w_e R_e S), S = floor(2^62/m) / max(w R)), so that the draws -- an integer
    decision -- are made from the same numbers on both sides; u holds the q uniform draws.
    Returns (count per edge, sparsifier conductance per edge)."""
    w = np.asarray(w, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    m = w.size
    s = w * R
    s = np.where(s > 0, s, 0.0)
    smax = s.max()
    scale_num = np.floor(np.ldexp(1.0, 62) / m)
    S = scale_num / smax if smax > 0 else 0.0
    k = np.floor(s * S).astype(np.int64)
    C = np.cumsum(k)
    K = int(C[-1])
    t = np.floor(u * np.float64(K)).astype(np.int64)
    t = np.clip(t, 0, K - 1)
    idx = np.searchsorted(C, t, side="right")          # first edge with C > t
    count = np.bincount(idx[idx < m], minlength=m).astype(np.int64)
    weight = np.zeros(m)
    nz = (count > 0) & (k > 0)
    weight[nz] = count[nz] * w[nz] * np.float64(K) / (np.float64(q) * k[nz].astype(np.float64))
    return count, weight
