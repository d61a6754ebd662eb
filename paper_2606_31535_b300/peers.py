"""Thin ctypes binding of libpeers.so (include/peers.h).

Argument marshalling only: every step of the computation runs in the library (host analysis
in C++, factorization and sweep in CUDA kernels).  PyTorch is used for device buffers and
the CUDA stream; the library is loaded from this package directory and a missing library is
an error, never a fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpeers.so")

OK = 0
EINVAL, ENOTCONNECTED, ENOTSPD, ENOMEM, ECUDA, ETIMEOUT, ENOTREADY = -1, -2, -3, -4, -5, -6, -7
OUT_DEVICE = 1

_lib = None


class PeersError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("ordering", ctypes.c_int32), ("nd_leaf", ctypes.c_int32),
                ("relax_small", ctypes.c_int32), ("relax_max", ctypes.c_int32),
                ("relax_frac", ctypes.c_double), ("carry_budget", ctypes.c_int64),
                ("qcap", ctypes.c_int32 * 4), ("front_smem", ctypes.c_int64),
                ("one_stream", ctypes.c_int64), ("reserved", ctypes.c_int64 * 4)]


class Stats(ctypes.Structure):
    _fields_ = [("sweep_s", ctypes.c_double), ("max_launch_s", ctypes.c_double),
                ("factor_s", ctypes.c_double), ("sweep_launches", ctypes.c_int64),
                ("factor_launches", ctypes.c_int64), ("h2d_bytes", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "failed", "queries",
                                               "steps", "launches", "peak_bytes")] + \
               [(k, ctypes.c_double) for k in ("wall_s", "qps", "p50_s", "p99_s", "mean_s")] + \
               [(k, ctypes.c_int64) for k in ("max_step_requests", "request_steps", "ready")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "n", "n_reduced", "nnz_a", "nnz_l", "nsuper", "levels", "max_nc", "max_nb", "nq",
        "nq_trivial", "nq_two_branch", "walk_entries", "walk_fma", "factor_fma",
        "device_bytes")] + [("t_order", ctypes.c_double), ("t_symbolic", ctypes.c_double),
                            ("t_queries", ctypes.c_double), ("nsuper_spilled", ctypes.c_int64),
                            ("front_bytes", ctypes.c_int64), ("lanes", ctypes.c_int64),
                            ("split_blocks", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def load(path: str | None = None):
    """Loads libpeers.so (or the library named by $PEERS_LIB, e.g. the bounds-checked
    libpeers_bounds.so); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("PEERS_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2606_31535_b300.build`")
    lib = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "peers_create": (ctypes.c_int, [P(vp), ctypes.c_int, vp]),
        "peers_destroy": (None, [vp]),
        "peers_analyze": (ctypes.c_int, [vp, i64, vp, vp, vp, i32, i64, vp, vp, vp, ctypes.c_int,
                                         vp, P(vp)]),
        "peers_symbolic_info": (ctypes.c_int, [vp, P(Info)]),
        "peers_num_queries": (i64, [vp]),
        "peers_footprint_bytes": (i64, [vp]),
        "peers_free_symbolic": (None, [vp]),
        "peers_symbolic_export": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
        "peers_factor": (ctypes.c_int, [vp, vp, vp, P(vp)]),
        "peers_numeric_diag": (ctypes.c_int, [vp, vp, vp]),
        "peers_free_numeric": (None, [vp]),
        "peers_query": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int]),
        "peers_query_noalloc": (ctypes.c_int, [vp, vp, vp, vp]),
        "peers_batch_create": (ctypes.c_int, [vp, ctypes.c_int32, vp, vp, ctypes.c_int, P(vp)]),
        "peers_batch_query": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "peers_batch_info": (ctypes.c_int, [vp, P(i64)]),
        "peers_batch_free": (None, [vp]),
        "peers_query_batch": (ctypes.c_int, [vp, ctypes.c_int32, vp, vp, vp, ctypes.c_int]),
        "peers_server_create": (ctypes.c_int, [ctypes.c_int, i64, ctypes.c_int32, ctypes.c_int32,
                                               vp, P(vp)]),
        "peers_server_submit": (ctypes.c_int, [vp, i64, vp, vp, vp, i32, i64, vp, vp, vp,
                                               ctypes.c_int, P(i64)]),
        "peers_server_poll": (ctypes.c_int, [vp, i64]),
        "peers_server_wait": (ctypes.c_int, [vp, i64, vp, i64, P(dbl)]),
        "peers_server_get_stats": (ctypes.c_int, [vp, P(ServerStats)]),
        "peers_server_hold": (ctypes.c_int, [vp, ctypes.c_int]),
        "peers_server_destroy": (None, [vp]),
        "peers_retile": (ctypes.c_int, [vp, vp, vp, vp]),
        "peers_query_blockinv": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int]),
        "peers_blockinv_bytes": (i64, [vp]),
        "peers_blockinv_fma": (i64, [vp]),
        "peers_query_selinv": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int]),
        "peers_sparsify": (ctypes.c_int, [vp, i64, vp, vp, i64, vp, vp, vp]),
        "peers_selinv_fma": (i64, [vp]),
        "peers_autotune": (ctypes.c_int, [vp, vp, vp, ctypes.c_char_p, vp, vp]),
        "peers_set_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "peers_last_stats": (ctypes.c_int, [vp, P(Stats)]),
        "peers_fp64_peak": (ctypes.c_int, [vp, P(dbl)]),
        "peers_last_level_times": (i64, [vp, P(dbl), i64]),
        "peers_fp64_mma_shapes": (ctypes.c_int, [vp, P(dbl)]),
        "peers_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "peers_last_error": (ctypes.c_char_p, []),
        "peers_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != OK:
        lib = load()
        msg = lib.peers_last_error().decode() or lib.peers_strerror(status).decode()
        raise PeersError(status, where, msg)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(int(a.data_ptr()))   # torch tensor


def _out_flags(ctx: "Context", out, n: int, where: str, device_only: bool = False) -> int:
    """Checks a result buffer before its pointer reaches the library (whose kernels write n
    doubles through it) and returns the matching flags: a writable, contiguous float64 numpy
    array of at least n entries (host), or a contiguous float64 torch CUDA tensor of at least
    n entries on the context's device."""
    if isinstance(out, np.ndarray):
        if device_only:
            raise ValueError(f"{where}: the result must be a CUDA tensor, not a numpy array")
        if out.dtype != np.float64 or not out.flags.c_contiguous or not out.flags.writeable \
                or out.size < n:
            raise ValueError(f"{where}: the host result must be a writable contiguous float64 "
                             f"array of at least {n} entries")
        return 0
    import torch
    if not isinstance(out, torch.Tensor):
        raise ValueError(f"{where}: the result must be a numpy array or a torch tensor")
    if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous() \
            or out.numel() < n:
        raise ValueError(f"{where}: the device result must be a contiguous float64 CUDA tensor "
                         f"of at least {n} entries")
    if out.device.index != ctx.device:
        raise ValueError(f"{where}: the result is on cuda:{out.device.index}, the context on "
                         f"cuda:{ctx.device}")
    return OUT_DEVICE


class Context:
    """A device and the CUDA stream the library issues its work on."""

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        self.device = device
        self._stream = stream
        handle = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        _check(lib.peers_create(ctypes.byref(handle), int(device), s), "peers_create")
        self._h = handle

    @classmethod
    def for_torch(cls, device: int = 0):
        """Context on torch's current stream of `device`."""
        import torch
        return cls(device, torch.cuda.current_stream(device))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().peers_destroy(self._h)
            self._h = None

    __del__ = close

    def set_timing(self, on: bool = True):
        _check(load().peers_set_timing(self._h, int(on)), "peers_set_timing")

    def last_stats(self) -> dict:
        st = Stats()
        _check(load().peers_last_stats(self._h, ctypes.byref(st)), "peers_last_stats")
        return st.as_dict()

    def fp64_peaks(self) -> dict:
        """Measured FP64 throughput (TFLOP/s): DFMA, mma.sync m8n8k4 f64, and both at once."""
        out = (ctypes.c_double * 3)()
        _check(load().peers_fp64_peak(self._h, out), "peers_fp64_peak")
        return {"dfma": out[0], "dmma": out[1], "dfma_with_dmma": out[2]}

    def fp64_mma_shapes(self) -> dict:
        """Measured FP64 tensor throughput (TFLOP/s) of every mma.sync .f64 shape."""
        out = (ctypes.c_double * 4)()
        _check(load().peers_fp64_mma_shapes(self._h, out), "peers_fp64_mma_shapes")
        return {"m8n8k4": out[0], "m16n8k4": out[1], "m16n8k8": out[2], "m16n8k16": out[3]}

    def last_level_times(self) -> np.ndarray:
        buf = (ctypes.c_double * 4096)()
        n = load().peers_last_level_times(self._h, buf, 4096)
        if n < 0:
            _check(n, "peers_last_level_times")
        return np.array(buf[:min(n, 4096)])


def _graph_args(n, indptr, indices, w, qu, qv, coords, where: str):
    """The graph, query and coordinate arrays in the library's types, with their sizes
    checked: the library reads n + 1 offsets, indptr[n] indices and conductances, nq query
    pairs and n x dim coordinates through plain pointers.  Returns
    (indptr, indices, w, qu, qv, nq, coords, dim), nq = -1 for all edges."""
    ip = np.ascontiguousarray(indptr, dtype=np.int64)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    wv = np.ascontiguousarray(w, dtype=np.float64)
    if int(n) < 0 or ip.ndim != 1 or ip.size != int(n) + 1:
        raise ValueError(f"{where}: indptr must hold n + 1 = {int(n) + 1} offsets")
    if ix.ndim != 1 or wv.ndim != 1 or ix.size != wv.size or ix.size != int(ip[-1]):
        raise ValueError(f"{where}: indices and w must each hold indptr[n] entries")
    nq = -1
    if qu is not None or qv is not None:
        if qu is None or qv is None:
            raise ValueError(f"{where}: qu and qv come together")
        qu = np.ascontiguousarray(qu, dtype=np.int32)
        qv = np.ascontiguousarray(qv, dtype=np.int32)
        if qu.ndim != 1 or qv.shape != qu.shape:
            raise ValueError(f"{where}: qu and qv must be 1-D and of one length")
        nq = qu.size
    c = None if coords is None else np.ascontiguousarray(coords, dtype=np.float64)
    dim = 0 if c is None else (c.shape[1] if c.ndim == 2 else 1)
    if c is not None and (c.ndim > 2 or c.size != int(n) * dim):
        raise ValueError(f"{where}: coords must be n x dim ({int(n)} x {dim})")
    return ip, ix, wv, qu, qv, nq, c, dim


class Symbolic:
    """Host plan: ordering, elimination tree, supernodes and query grouping."""

    def __init__(self, n, indptr, indices, w, ground=0, qu=None, qv=None, coords=None,
                 options: Options | None = None):
        lib = load()
        ip, ix, wv, qu, qv, nq, c, dim = _graph_args(n, indptr, indices, w, qu, qv, coords,
                                                     "peers_analyze")
        self._keep = [ip, ix, wv]
        h = ctypes.c_void_p()
        opt = ctypes.byref(options) if options is not None else None
        _check(lib.peers_analyze(None, int(n), _ptr(self._keep[0]), _ptr(self._keep[1]),
                                 _ptr(self._keep[2]), int(ground), int(nq), _ptr(qu), _ptr(qv),
                                 _ptr(c), int(dim), opt, ctypes.byref(h)), "peers_analyze")
        self._h = h
        self.n = int(n)
        self.nnz = int(ix.size)
        self.nq = int(lib.peers_num_queries(h))

    @classmethod
    def of(cls, g, ground=0, qu=None, qv=None, use_coords=True, options=None):
        return cls(g.n, g.indptr, g.indices, g.w, ground, qu, qv,
                   g.coords if use_coords else None, options)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().peers_free_symbolic(self._h)
            self._h = None

    __del__ = close

    def info(self) -> dict:
        inf = Info()
        _check(load().peers_symbolic_info(self._h, ctypes.byref(inf)), "peers_symbolic_info")
        return inf.as_dict()

    def footprint_bytes(self) -> int:
        return int(load().peers_footprint_bytes(self._h))

    def export(self) -> dict:
        inf = self.info()
        nr, ns = inf["n_reduced"], inf["nsuper"]
        perm = np.empty(nr, np.int32)
        first = np.empty(ns + 1, np.int32)
        parent = np.empty(ns, np.int32)
        nb = np.empty(ns, np.int32)
        level = np.empty(ns, np.int32)
        _check(load().peers_symbolic_export(self._h, _ptr(perm), _ptr(first), _ptr(parent),
                                            _ptr(nb), _ptr(level)), "peers_symbolic_export")
        return {"perm": perm, "first": first, "parent": parent, "nb": nb, "level": level}


class Numeric:
    """Device-resident L D L^T factor of a plan's grounded Laplacian."""

    def __init__(self, ctx: Context, sym: Symbolic, w=None):
        lib = load()
        self._ctx, self._sym = ctx, sym
        self._w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        if self._w is not None and (self._w.ndim != 1 or self._w.size != sym.nnz):
            raise ValueError(f"peers_factor: w must hold one conductance per stored CSR entry "
                             f"({sym.nnz})")
        h = ctypes.c_void_p()
        _check(lib.peers_factor(ctx._h, sym._h, _ptr(self._w), ctypes.byref(h)), "peers_factor")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().peers_free_numeric(self._h)
            self._h = None

    __del__ = close

    def diag(self) -> np.ndarray:
        d = np.empty(self._sym.info()["n_reduced"], np.float64)
        _check(load().peers_numeric_diag(self._ctx._h, self._h, _ptr(d)), "peers_numeric_diag")
        return d


def query_blockinv(ctx: Context, sym: Symbolic, num: Numeric, out=None):
    """Resistances of the plan's queries through the block implicit inverse (the paper's order
    of work); same interface as :func:`query`."""
    lib = load()
    if out is None:
        out = np.empty(sym.nq, dtype=np.float64)
    flags = _out_flags(ctx, out, sym.nq, "query_blockinv")
    _check(lib.peers_query_blockinv(ctx._h, sym._h, num._h, _ptr(out), flags),
           "peers_query_blockinv")
    return out


def query_selinv(ctx: Context, sym: Symbolic, num: Numeric, out=None):
    """Resistances of the plan's queries from the selected inverse (edges and pairs touching
    the ground only); same interface as :func:`query`."""
    lib = load()
    if out is None:
        out = np.empty(sym.nq, dtype=np.float64)
    flags = _out_flags(ctx, out, sym.nq, "query_selinv")
    _check(lib.peers_query_selinv(ctx._h, sym._h, num._h, _ptr(out), flags), "peers_query_selinv")
    return out


def sparsify(ctx: Context, w, R, u):
    """Alg. 1 on the device: w, R (m) and u (q uniforms) are float64 CUDA tensors; returns
    (count int64, weight float64) CUDA tensors of m entries."""
    import torch

    def device_f64(t, name, n=None):
        # the kernels read every entry through the raw pointer: a contiguous float64 CUDA
        # tensor on the context's device, of the stated length
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda \
                or not t.is_contiguous() or t.dim() != 1 or (n is not None and t.numel() != n):
            raise ValueError(f"sparsify: {name} must be a contiguous 1-D float64 CUDA tensor"
                             + ("" if n is None else f" of {n} entries"))
        if t.device.index != ctx.device:
            raise ValueError(f"sparsify: {name} is on cuda:{t.device.index}, the context on "
                             f"cuda:{ctx.device}")

    device_f64(w, "w")
    m = int(w.numel())
    device_f64(R, "R", m)
    device_f64(u, "u")
    q = int(u.numel())
    count = torch.empty(m, dtype=torch.int64, device=w.device)
    weight = torch.empty(m, dtype=torch.float64, device=w.device)
    _check(load().peers_sparsify(ctx._h, m, _ptr(w), _ptr(R), q, _ptr(u), _ptr(count),
                                 _ptr(weight)), "peers_sparsify")
    return count, weight


def blockinv_cost(sym: Symbolic) -> dict:
    lib = load()
    return {"bytes": int(lib.peers_blockinv_bytes(sym._h)), "fma": int(lib.peers_blockinv_fma(sym._h))}


def retile(ctx: Context, sym: Symbolic, num: Numeric, qcap):
    """Re-tiles a factored plan with per-size-class caps (4 ints; 0 = largest that fits)."""
    caps = np.ascontiguousarray(qcap, dtype=np.int32)
    _check(load().peers_retile(ctx._h, sym._h, num._h, _ptr(caps)), "peers_retile")


def autotune(ctx: Context, sym: Symbolic, num: Numeric, cache_path: str | None = None) -> dict:
    """Times the candidate tile caps per front-size class on this plan, re-tiles it with the
    fastest, and records them in `cache_path`.  Returns {"qcap": [...], "gain": [...]}."""
    caps = np.zeros(4, dtype=np.int32)
    gain = np.zeros(4, dtype=np.float64)
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(load().peers_autotune(ctx._h, sym._h, num._h, path, _ptr(caps), _ptr(gain)),
           "peers_autotune")
    return {"qcap": caps.tolist(), "gain": gain.tolist()}


def query(ctx: Context, sym: Symbolic, num: Numeric, out=None):
    """Resistances of the plan's queries.  `out` may be a float64 torch CUDA tensor (written on
    the device) or a numpy array (host); None allocates a numpy array."""
    lib = load()
    if out is None:
        out = np.empty(sym.nq, dtype=np.float64)
    flags = _out_flags(ctx, out, sym.nq, "query")
    _check(lib.peers_query(ctx._h, sym._h, num._h, _ptr(out), flags), "peers_query")
    return out


BATCH_CUDA_GRAPH = 1


class Batch:
    """Many factored graphs swept together: one persistent launch per aligned etree level,
    optionally captured in a CUDA graph (replayed on every query after the first)."""

    def __init__(self, ctx: Context, syms, nums, cuda_graph: bool = True):
        lib = load()
        self._ctx, self._syms, self._nums = ctx, list(syms), list(nums)
        n = len(self._syms)
        hs = (ctypes.c_void_p * n)(*[s._h.value for s in self._syms])
        hn = (ctypes.c_void_p * n)(*[m._h.value for m in self._nums])
        h = ctypes.c_void_p()
        _check(lib.peers_batch_create(ctx._h, n, hs, hn, BATCH_CUDA_GRAPH if cuda_graph else 0,
                                      ctypes.byref(h)), "peers_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().peers_batch_free(self._h)
            self._h = None

    __del__ = close

    def info(self) -> dict:
        out = (ctypes.c_int64 * 4)()
        _check(load().peers_batch_info(self._h, out), "peers_batch_info")
        return {"steps": out[0], "items": out[1], "launches": out[2], "device_bytes": out[3]}

    def query(self, outs=None):
        """Returns (or fills) one result array per graph: numpy arrays (host) or float64 torch
        CUDA tensors (device)."""
        if outs is None:
            outs = [np.empty(s.nq, dtype=np.float64) for s in self._syms]
        n = len(outs)
        if n != len(self._syms):
            raise ValueError("Batch.query: one result buffer per graph")
        flags = {_out_flags(self._ctx, o, s.nq, "Batch.query") for o, s in zip(outs, self._syms)}
        if len(flags) != 1:
            raise ValueError("Batch.query: all results on the host or all on the device")
        flags = flags.pop()
        ptrs = (ctypes.c_void_p * n)(*[_ptr(o).value for o in outs])
        _check(load().peers_batch_query(self._ctx._h, self._h, ptrs, flags), "peers_batch_query")
        return outs


class Server:
    """Continuous-batching request loop on one device (see peers_server_* in peers.h)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, max_active: int = 0,
                 workers: int = 0, options: Options | None = None):
        lib = load()
        h = ctypes.c_void_p()
        self._opt = options
        opt = ctypes.byref(options) if options is not None else None
        _check(lib.peers_server_create(int(device), int(mem_budget_bytes), int(max_active),
                                       int(workers), opt, ctypes.byref(h)), "peers_server_create")
        self._h = h
        self._nq = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().peers_server_destroy(self._h)
            self._h = None

    __del__ = close

    def submit(self, g, qu=None, qv=None, ground: int = 0, use_coords: bool = True) -> int:
        """Queues a request (graph + queries; all edges when qu is None); returns its ticket.
        The library copies the arrays before returning."""
        ip, ix, w, qu, qv, nq, c, dim = _graph_args(
            g.n, g.indptr, g.indices, g.w, qu, qv, g.coords if use_coords else None,
            "peers_server_submit")
        t = ctypes.c_int64()
        _check(load().peers_server_submit(self._h, int(g.n), _ptr(ip), _ptr(ix), _ptr(w),
                                          int(ground), int(nq), _ptr(qu), _ptr(qv), _ptr(c), dim,
                                          ctypes.byref(t)), "peers_server_submit")
        self._nq[t.value] = g.m if nq < 0 else nq
        return t.value

    def poll(self, ticket: int) -> int:
        return int(load().peers_server_poll(self._h, int(ticket)))

    def wait(self, ticket: int):
        """(results, latency seconds) of a request; raises PeersError if it failed."""
        nq = self._nq.pop(ticket)
        R = np.empty(nq, dtype=np.float64)
        lat = ctypes.c_double()
        _check(load().peers_server_wait(self._h, int(ticket), _ptr(R), nq, ctypes.byref(lat)),
               "peers_server_wait")
        return R, lat.value

    def hold(self, on: bool = True):
        """While held, factored requests wait instead of joining the sweep (stats()["ready"]
        counts them); releasing lets them all join at the next step."""
        _check(load().peers_server_hold(self._h, int(on)), "peers_server_hold")

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().peers_server_get_stats(self._h, ctypes.byref(st)), "peers_server_get_stats")
        return st.as_dict()


def query_noalloc(ctx: Context, sym: Symbolic, num: Numeric, out):
    """Resistances into the device tensor `out` (float64, sym.nq entries) with the library's
    static scratch array: the library allocates no device memory during the call."""
    _out_flags(ctx, out, sym.nq, "query_noalloc", device_only=True)
    _check(load().peers_query_noalloc(ctx._h, sym._h, num._h, _ptr(out)), "peers_query_noalloc")
    return out


def effective_resistance(g, qu=None, qv=None, ground=0, device=0, use_coords=True):
    """One-shot convenience: analyse, factor on `device` and sweep; returns a numpy array."""
    ctx = Context(device)
    sym = Symbolic.of(g, ground, qu, qv, use_coords)
    num = Numeric(ctx, sym)
    return query(ctx, sym, num)
