"""Thin Python binding of libssg.so (the C ABI declared in include/ssg.h).

Argument marshalling only: every step of the NSSG build and search runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors; the calls run on the current torch
stream.  There is no CPU fallback: if libssg.so is missing or cannot load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libssg.so")
_lock = threading.Lock()
_lib = None

PREC = {"fp32": 0, "bf16": 1, "auto": 2, "bf16_rerank": 3, "fp8": 4}


class SSGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ssg status {status}: {msg}")
        self.status = status


class BuildOpts(ctypes.Structure):
    _fields_ = [("gemm_prec", ctypes.c_int), ("n_nav", ctypes.c_int32),
                ("nav_ids_host", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("debug_checks", ctypes.c_int32), ("pool_tiles", ctypes.c_int32),
                ("pool_own_row_first", ctypes.c_int32), ("gram_prec", ctypes.c_int),
                ("cos_margin_fp64", ctypes.c_double), ("tune_table", ctypes.c_char_p)]


class BuildStats(ctypes.Structure):
    _fields_ = [("ms_ingest", ctypes.c_double), ("ms_knn", ctypes.c_double),
                ("ms_pool", ctypes.c_double), ("ms_prune", ctypes.c_double),
                ("ms_reverse", ctypes.c_double), ("ms_connect", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("n_repair", ctypes.c_int64),
                ("n_angle_fp64", ctypes.c_int64), ("n_order_fp64", ctypes.c_int64),
                ("n_knn_fallback_rows", ctypes.c_int64), ("max_indegree", ctypes.c_int32),
                ("exact_mode", ctypes.c_int32), ("kernel_launches", ctypes.c_int64),
                ("gemm_prec_used", ctypes.c_int32), ("ms_knn_gemm", ctypes.c_double),
                ("search_row_bytes", ctypes.c_int32), ("gram_prec_used", ctypes.c_int32),
                ("n_angle_borderline", ctypes.c_int64), ("knn_candidates", ctypes.c_int32),
                ("ms_knn_certify", ctypes.c_double), ("n_repair_knn_row", ctypes.c_int64),
                ("knn_bf16_pairs", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SYMBOLS = {
    # name: (restype, argtypes)
    "ssg_selftest_wait": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_debug_fail_alloc": (None, [ctypes.c_int64]),
    "ssg_check_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "ssg_default_opts": (None, [ctypes.c_void_p]),
    "ssg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "ssg_last_error": (ctypes.c_char_p, []),
    "ssg_last_device_status": (ctypes.c_int, []),
    "ssg_kernel_launch_count": (ctypes.c_int64, []),
    "ssg_nav_ids": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p]),
    "ssg_knn": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_knn_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_pool": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_prune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_reverse": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "ssg_connect": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "ssg_connect_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "ssg_search_adj": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_search_work": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "ssg_recall_hits": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_build_batched": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_autotune_batched": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_char_p, ctypes.c_void_p]),
    "ssg_build_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "ssg_graph_view": (ctypes.c_int, [ctypes.c_void_p] * 8),
    "ssg_search": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_search_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_server_default_opts": (None, [ctypes.c_void_p]),
    "ssg_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "ssg_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "ssg_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "ssg_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_server_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ssg_server_destroy": (None, [ctypes.c_void_p]),
    "ssg_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "ssg_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_void_p]),
    "ssg_free": (None, [ctypes.c_void_p]),
}


def lib():
    """Load libssg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_1907_06146_gb300.build_ext.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SYMBOLS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(status: int):
    if status != 0:
        msg = lib().ssg_last_error().decode(errors="replace")
        raise SSGError(status, msg)


def launch_count() -> int:
    return int(lib().ssg_kernel_launch_count())


def nav_ids(n: int, s: int, seed: int) -> np.ndarray:
    out = np.empty(s, np.int32)
    _check(lib().ssg_nav_ids(n, s, seed, out.ctypes.data_as(ctypes.c_void_p)))
    return out


# ---- torch marshalling ----------------------------------------------------------------
def _torch():
    import torch
    return torch


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _dev(t, dtype):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t))
    t = t.to(device="cuda", dtype=dtype)
    return t.contiguous()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def check_graph(adj, deg):
    """Invariant check of a device adjacency (ssg_check_graph): (bad row or -1, code)."""
    torch = _torch()
    a = _dev(adj, torch.int32)
    dg = _dev(deg, torch.int32)
    row = ctypes.c_int64()
    code = ctypes.c_int32()
    _check(lib().ssg_check_graph(_ptr(a), _ptr(dg), a.shape[0], a.shape[1], ctypes.byref(row),
                                 ctypes.byref(code), _stream()))
    return int(row.value), int(code.value)


def last_device_status() -> int:
    """Status of the latest failure a kernel reported on the device (0 if none); clears it
    (ssg_last_device_status)."""
    return int(lib().ssg_last_device_status())


def debug_fail_alloc(nth: int):
    """Fault injection on the host: the nth scratch allocation from now on fails (ENOMEM);
    0 switches it off (ssg_debug_fail_alloc)."""
    lib().ssg_debug_fail_alloc(int(nth))


def selftest_wait(mode: int):
    """The bounded-wait self-test (ssg_selftest_wait): returns (wait succeeded, elapsed ms)."""
    ok = ctypes.c_int32()
    ms = ctypes.c_int32()
    _check(lib().ssg_selftest_wait(mode, ctypes.byref(ok), ctypes.byref(ms)))
    return bool(ok.value), int(ms.value)


def knn(base, K: int, prec: str = "auto"):
    """Exact kNN graph: (ids int32 [n][K], d2 float32 [n][K])."""
    torch = _torch()
    b = _dev(base, torch.float32)
    n, d = b.shape
    ids = torch.empty((n, K), dtype=torch.int32, device="cuda")
    d2 = torch.empty((n, K), dtype=torch.float32, device="cuda")
    _check(lib().ssg_knn(_ptr(b), n, d, K, PREC[prec], _ptr(ids), _ptr(d2), _stream()))
    return ids, d2


def knn_query(base, queries, k: int, prec: str = "auto"):
    """Brute-force ground truth: (ids int32 [nq][k], d2 float32 [nq][k])."""
    torch = _torch()
    b = _dev(base, torch.float32)
    q = _dev(queries, torch.float32)
    n, d = b.shape
    nq = q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    _check(lib().ssg_knn_query(_ptr(b), n, d, _ptr(q), nq, k, PREC[prec], _ptr(ids), _ptr(d2),
                               _stream()))
    return ids, d2


def pool(base, knn_id, L: int):
    torch = _torch()
    b = _dev(base, torch.float32)
    kn = _dev(knn_id, torch.int32)
    n, d = b.shape
    K = kn.shape[1]
    pid = torch.empty((n, L), dtype=torch.int32, device="cuda")
    pd2 = torch.empty((n, L), dtype=torch.float32, device="cuda")
    pl = torch.empty((n,), dtype=torch.int32, device="cuda")
    _check(lib().ssg_pool(_ptr(b), n, d, _ptr(kn), K, L, _ptr(pid), _ptr(pd2), _ptr(pl), _stream()))
    return pid, pd2, pl


def prune(base, pool_id, pool_len, R: int, alpha: float):
    torch = _torch()
    b = _dev(base, torch.float32)
    pid = _dev(pool_id, torch.int32)
    pl = _dev(pool_len, torch.int32)
    n, d = b.shape
    adj = torch.empty((n, R), dtype=torch.int32, device="cuda")
    deg = torch.empty((n,), dtype=torch.int32, device="cuda")
    _check(lib().ssg_prune(_ptr(b), n, d, _ptr(pid), _ptr(pl), pid.shape[1], R, float(alpha),
                           _ptr(adj), _ptr(deg), _stream()))
    return adj, deg


def reverse(base, adj0, deg0, alpha: float):
    torch = _torch()
    b = _dev(base, torch.float32)
    a0 = _dev(adj0, torch.int32)
    d0 = _dev(deg0, torch.int32)
    n, d = b.shape
    R = a0.shape[1]
    adj1 = torch.empty_like(a0)
    deg1 = torch.empty_like(d0)
    _check(lib().ssg_reverse(_ptr(b), n, d, _ptr(a0), _ptr(d0), R, float(alpha), _ptr(adj1),
                             _ptr(deg1), _stream()))
    return adj1, deg1


def connect(base, adj, deg, nav):
    """Connectivity repair on copies of adj/deg; returns (adj, deg, n_repair)."""
    torch = _torch()
    b = _dev(base, torch.float32)
    a = _dev(adj, torch.int32).clone()
    dg = _dev(deg, torch.int32).clone()
    nv = _dev(nav, torch.int32)
    n, d = b.shape
    rep = ctypes.c_int64(0)
    _check(lib().ssg_connect(_ptr(b), n, d, _ptr(a), _ptr(dg), a.shape[1], _ptr(nv), nv.numel(),
                             ctypes.byref(rep), _stream()))
    return a, dg, int(rep.value)


def search_adj(base, adj, deg, nav, queries, k: int, L_search: int):
    torch = _torch()
    b = _dev(base, torch.float32)
    a = _dev(adj, torch.int32)
    dg = _dev(deg, torch.int32)
    nv = _dev(nav, torch.int32)
    q = _dev(queries, torch.float32)
    n, d = b.shape
    nq = q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    _check(lib().ssg_search_adj(_ptr(b), n, d, _ptr(a), _ptr(dg), a.shape[1], _ptr(nv), nv.numel(),
                                _ptr(q), nq, k, L_search, _ptr(ids), _ptr(d2), _stream()))
    return ids, d2


def search_work(base, adj, deg, nav, queries, k: int, L_search: int):
    """search_adj plus the batch's work: {expansions, distances, adjacency_entries}."""
    torch = _torch()
    b = _dev(base, torch.float32)
    a = _dev(adj, torch.int32)
    dg = _dev(deg, torch.int32)
    nv = _dev(nav, torch.int32)
    q = _dev(queries, torch.float32)
    n, d = b.shape
    nq = q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    w = (ctypes.c_int64 * 3)()
    _check(lib().ssg_search_work(_ptr(b), n, d, _ptr(a), _ptr(dg), a.shape[1], _ptr(nv),
                                 nv.numel(), _ptr(q), nq, k, L_search, _ptr(ids), _ptr(d2), w,
                                 _stream()))
    return ids, d2, {"expansions": w[0], "distances": w[1], "adjacency_entries": w[2]}


def recall_hits(found, truth, k: int) -> int:
    torch = _torch()
    f = _dev(found, torch.int32)
    t = _dev(truth, torch.int32)
    h = ctypes.c_int64(0)
    _check(lib().ssg_recall_hits(_ptr(f), f.shape[1], _ptr(t), t.shape[1], f.shape[0], k,
                                 ctypes.byref(h), _stream()))
    return int(h.value)


class _DevView:
    """A device array owned by the library, exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": tuple(shape),
                                         "typestr": typestr, "version": 2, "strides": None}
        self._owner = owner


class Graph:
    """An NSSG index owned by the library (released on garbage collection)."""

    def __init__(self, handle: ctypes.c_void_p, stats: BuildStats | None = None):
        self._h = handle
        self.stats = stats.as_dict() if stats is not None else None
        adj, deg, nav = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        n_nav, R, d = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        n = ctypes.c_int64()
        _check(lib().ssg_graph_view(self._h, ctypes.byref(adj), ctypes.byref(deg), ctypes.byref(nav),
                                    ctypes.byref(n_nav), ctypes.byref(R), ctypes.byref(n),
                                    ctypes.byref(d)))
        self.n, self.d, self.R, self.n_nav = n.value, d.value, R.value, n_nav.value
        self._adj, self._deg, self._nav = adj.value, deg.value, nav.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ssg_free(self._h)
            self._h = None

    def _view(self, ptr, shape):
        torch = _torch()
        return torch.as_tensor(_DevView(ptr, shape, "<i4", self), device="cuda")

    @property
    def adj(self):
        return self._view(self._adj, (self.n, self.R))

    @property
    def deg(self):
        return self._view(self._deg, (self.n,))

    @property
    def nav(self):
        return self._view(self._nav, (self.n_nav,))

    def search(self, base, queries, k: int, L_search: int):
        torch = _torch()
        q = _dev(queries, torch.float32)
        b = ctypes.c_void_p(0) if base is None else _ptr(_dev(base, torch.float32))
        nq = q.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
        d2 = torch.empty((nq, k), dtype=torch.float32, device="cuda")
        _check(lib().ssg_search(self._h, b, _ptr(q), nq, k, L_search, _ptr(ids), _ptr(d2), _stream()))
        return ids, d2

    def search_host(self, queries: np.ndarray, k: int, L_search: int):
        """Alg. 1 with host queries and host results (copies inside the call)."""
        q = np.ascontiguousarray(queries, dtype=np.float32)
        ids = np.empty((q.shape[0], k), np.int32)
        d2 = np.empty((q.shape[0], k), np.float32)
        _check(lib().ssg_search_host(self._h, q.ctypes.data_as(ctypes.c_void_p), q.shape[0], k,
                                     L_search, ids.ctypes.data_as(ctypes.c_void_p),
                                     d2.ctypes.data_as(ctypes.c_void_p), _stream()))
        return ids, d2

    def save(self, path: str):
        _check(lib().ssg_save(self._h, path.encode()))

    @staticmethod
    def load(path: str) -> "Graph":
        h = ctypes.c_void_p()
        _check(lib().ssg_load(path.encode(), ctypes.byref(h)))
        return Graph(h)


class ServerOpts(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_int64), ("max_k", ctypes.c_int32),
                ("max_L_search", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_int64), ("queries_done", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("max_batches_in_flight", ctypes.c_int64),
                ("max_queries_in_flight", ctypes.c_int64), ("busy_ms", ctypes.c_double)]


class Server:
    """Continuous-batching search server over a built graph (see ssg_server_* in ssg.h).
    submit() returns a ticket at once; wait(ticket) blocks and returns (ids, d2, latency_ms).
    Safe to call from several host threads."""

    def __init__(self, graph: Graph, base=None, n_streams: int = 4, max_batch: int = 8192,
                 mem_budget_bytes: int = 256 << 20, max_k: int = 128, max_L_search: int = 1024):
        o = ServerOpts()
        lib().ssg_server_default_opts(ctypes.byref(o))
        o.n_streams, o.max_batch, o.mem_budget_bytes = n_streams, max_batch, mem_budget_bytes
        o.max_k, o.max_L_search = max_k, max_L_search
        self._graph = graph
        self._base = None if base is None else _dev(base, _torch().float32)
        bp = ctypes.c_void_p(0) if self._base is None else _ptr(self._base)
        self._h = ctypes.c_void_p()
        _check(lib().ssg_server_create(graph._h, bp, ctypes.byref(o), ctypes.byref(self._h)))
        self._shape = {}
        self._lock = __import__("threading").Lock()

    def submit(self, queries: np.ndarray, k: int, L_search: int) -> int:
        q = np.ascontiguousarray(queries, dtype=np.float32)
        t = ctypes.c_uint64()
        _check(lib().ssg_server_submit(self._h, q.ctypes.data_as(ctypes.c_void_p), q.shape[0], k,
                                       L_search, ctypes.byref(t)))
        with self._lock:
            self._shape[t.value] = (q.shape[0], k)
        return t.value

    def wait(self, ticket: int):
        with self._lock:
            nq, k = self._shape.pop(ticket)
        ids = np.empty((nq, k), np.int32)
        d2 = np.empty((nq, k), np.float32)
        lat = ctypes.c_double()
        _check(lib().ssg_server_wait(self._h, ticket, ids.ctypes.data_as(ctypes.c_void_p),
                                     d2.ctypes.data_as(ctypes.c_void_p), ctypes.byref(lat)))
        return ids, d2, lat.value

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().ssg_server_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().ssg_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _opts(n_nav, nav, seed, prec, gram_prec="auto", cos_margin=None, tune_table=None):
    o = BuildOpts()
    lib().ssg_default_opts(ctypes.byref(o))
    o.gemm_prec = PREC[prec]
    o.gram_prec = PREC[gram_prec]
    if cos_margin is not None:
        o.cos_margin_fp64 = float(cos_margin)
    if tune_table is not None:
        o.tune_table = tune_table.encode() if isinstance(tune_table, str) else tune_table
    keep = None
    if nav is not None:
        keep = np.ascontiguousarray(np.asarray(nav), dtype=np.int32)
        o.n_nav = keep.size
        o.nav_ids_host = keep.ctypes.data
    else:
        o.n_nav = n_nav
    if seed is not None:
        o.seed = seed
    return o, keep


def build(base, K: int, L: int, R: int, alpha: float, n_nav: int = 10, nav=None, seed=None,
          prec: str = "auto", pool_tiles: int = 0, pool_own_row_first: bool = False,
          debug_checks: bool = False, gram_prec: str = "auto", cos_margin=None,
          tune_table=None) -> Graph:
    """NSSGIndexing on a device-resident base (torch CUDA float32 [n][d]): Alg. 3, or with
    pool_tiles > 0 Alg. 4's pools searched on the fly over the cluster-ordered tiles.
    prec / gram_prec: arithmetic of the kNN GEMM and of the prune's Gram (the graph is the
    same for every choice); cos_margin: the angle test's reporting band (default 1e-5);
    tune_table: path of a launch-parameter file."""
    torch = _torch()
    b = _dev(base, torch.float32)
    n, d = b.shape
    o, keep = _opts(n_nav, nav, seed, prec, gram_prec, cos_margin, tune_table)
    o.pool_tiles = pool_tiles
    o.pool_own_row_first = int(pool_own_row_first)
    o.debug_checks = int(debug_checks)
    h = ctypes.c_void_p()
    st = BuildStats()
    _check(lib().ssg_build(_ptr(b), n, d, K, L, R, float(alpha), ctypes.byref(o), _stream(),
                           ctypes.byref(h), ctypes.byref(st)))
    del keep
    g = Graph(h, st)
    g._base_ref = b
    return g


def _batch_args(bases, K, L, R, alpha):
    torch = _torch()
    bs = [_dev(b, torch.float32) for b in bases]
    m = len(bs)

    def per(v, ctype):
        vals = list(v) if isinstance(v, (list, tuple)) else [v] * m
        return (ctype * m)(*vals)

    ptrs = (ctypes.c_void_p * m)(*[_ptr(b) for b in bs])
    ns = (ctypes.c_int64 * m)(*[b.shape[0] for b in bs])
    ds = (ctypes.c_int32 * m)(*[b.shape[1] for b in bs])
    return (bs, m, ptrs, ns, ds, per(K, ctypes.c_int32), per(L, ctypes.c_int32),
            per(R, ctypes.c_int32), per(alpha, ctypes.c_double))


def autotune_batched(bases, K, L, R, alpha, path: str, n_nav: int = 10, seed=None,
                     prec: str = "auto"):
    """Times the batched build's launch parameters on the batch's largest indices and writes
    the fastest as a tune-table file at path (ssg_autotune_batched); returns (best batched
    prune ms, best kNN ms)."""
    torch = _torch()
    bs, m, ptrs, ns, ds, Ks, Ls, Rs, As = _batch_args(bases, K, L, R, alpha)
    o, keep = _opts(n_nav, None, seed, prec)
    best = (ctypes.c_double * 2)()
    torch.cuda.synchronize()
    _check(lib().ssg_autotune_batched(m, ptrs, ns, ds, Ks, Ls, Rs, As, ctypes.byref(o),
                                      path.encode(), best))
    del keep
    return best[0], best[1]


def build_batched(bases, K, L, R, alpha, n_nav: int = 10, seed=None, prec: str = "auto",
                  n_streams: int = 8, tune_table=None):
    """Independent indices built concurrently (ssg_build_batched): bases is a list of
    device float32 [n_i][d_i] tensors; K, L, R, alpha are scalars or per-index lists.
    Returns the list of Graphs (each equal to ssg_build's for the same input)."""
    torch = _torch()
    bs, m, ptrs, ns, ds, Ks, Ls, Rs, As = _batch_args(bases, K, L, R, alpha)
    o, keep = _opts(n_nav, None, seed, prec, tune_table=tune_table)
    hs = (ctypes.c_void_p * m)()
    sts = (BuildStats * m)()
    torch.cuda.synchronize()  # the inputs are read on the library's own streams
    _check(lib().ssg_build_batched(m, ptrs, ns, ds, Ks, Ls, Rs, As, ctypes.byref(o), n_streams,
                                   hs, sts))
    del keep
    out = []
    for i in range(m):
        g = Graph(ctypes.c_void_p(hs[i]), sts[i])
        g._base_ref = bs[i]
        out.append(g)
    return out


def build_host(base: np.ndarray, K: int, L: int, R: int, alpha: float, n_nav: int = 10, nav=None,
               seed=None, prec: str = "auto", adj_out=None, deg_out=None):
    """NSSGIndexing from host vectors; returns (graph, adj numpy [n][R], deg numpy [n]).
    adj_out / deg_out: optional int32 C-contiguous host arrays of those shapes to receive the
    graph (pinned memory makes the copy back faster)."""
    x = np.ascontiguousarray(base, dtype=np.float32)
    n, d = x.shape
    o, keep = _opts(n_nav, nav, seed, prec)
    adj = adj_out if adj_out is not None else np.empty((n, R), np.int32)
    deg = deg_out if deg_out is not None else np.empty(n, np.int32)
    if (adj.shape != (n, R) or deg.shape != (n,) or adj.dtype != np.int32
            or deg.dtype != np.int32 or not adj.flags.c_contiguous or not deg.flags.c_contiguous):
        raise ValueError("adj_out must be int32 [n][R] and deg_out int32 [n], C-contiguous")
    h = ctypes.c_void_p()
    st = BuildStats()
    _check(lib().ssg_build_host(x.ctypes.data_as(ctypes.c_void_p), n, d, K, L, R, float(alpha),
                                ctypes.byref(o), _stream(), ctypes.byref(h),
                                adj.ctypes.data_as(ctypes.c_void_p),
                                deg.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st)))
    del keep
    return Graph(h, st), adj, deg
