"""CPU oracle for the NSSG hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The CUDA library never calls it, and it imports nothing
from the CUDA package.  The arithmetic lives in ``nssg_oracle.c`` (double precision,
sequential sums, no fused multiply-add); this module compiles it with gcc on first use
and wraps it with numpy arrays.

Every function follows the passage of the paper (arXiv 1907.06146) that its docstring
names; readings R1..R13 where the paper is silent or garbled are stated in the C source.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (hand-derived fixtures, library routines, definitions and
theorems of the paper); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nssg_oracle.c")
_LIB = os.path.join(_HERE, "libnssg_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
          "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU, no CUDA) into oracle/libnssg_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.or_knn_rows.argtypes = [P, i64, i32, P, i64, i32, P, P]
        lib.or_knn_queries.argtypes = [P, i64, i32, P, i64, i32, P, P]
        lib.or_pool.argtypes = [P, i64, i32, P, i32, i32, P, i64, P, P, P]
        lib.or_pool2.argtypes = [P, i64, i32, P, i32, i32, P, i64, i32, P, P, P]
        lib.or_prune.argtypes = [P, i64, i32, P, i64, P, P, i32, i32, dbl, P, P]
        lib.or_reverse.argtypes = [P, i64, i32, P, P, i32, dbl, P, P]
        lib.or_connect.argtypes = [P, i64, i32, P, P, i32, P, i32, P]
        lib.or_search.argtypes = [P, i64, i32, P, P, i32, P, i32, P, i64, i32, i32, P, P, P, P]
        lib.or_dist2_pairs.argtypes = [P, i32, P, P, i64, P]
        lib.or_cos_triples.argtypes = [P, i32, P, P, P, i64, P]
        lib.or_set_threads.argtypes = [i32]
        lib.or_max_threads.restype = i32
        _lib = lib
        return lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().or_max_threads())


def set_threads(t: int) -> None:
    _load().or_set_threads(int(t))


def cos_alpha(alpha_deg: float) -> float:
    """cos of the angle alpha given in degrees.  Angles whose cosine is rational (0, 60,
    90, 120, 180 degrees) use that exact value, so that e.g. the 60-degree test is
    exactly cos > 1/2; other angles use the C library cosine."""
    exact = {0.0: 1.0, 60.0: 0.5, 90.0: 0.0, 120.0: -0.5, 180.0: -1.0}
    a = float(alpha_deg)
    if a in exact:
        return exact[a]
    return math.cos(a * math.pi / 180.0)


def knn_rows(base, K, rows=None):
    """Exact K nearest neighbours of the given base rows (all rows if None), self
    excluded, ordered by (d2, id).  Returns (ids int32 [m][K], d2 float64 [m][K])."""
    base = _f32(base)
    n, d = base.shape
    rows = _i64(np.arange(n) if rows is None else rows)
    ids = np.empty((rows.size, K), np.int32)
    d2 = np.empty((rows.size, K), np.float64)
    rc = _load().or_knn_rows(_p(base), n, d, _p(rows), rows.size, K, _p(ids), _p(d2))
    if rc != 0:
        raise ValueError("K must be < n")
    return ids, d2


def knn_queries(base, queries, k):
    """Brute-force ground truth: the k base points nearest each query by (d2, id)."""
    base, queries = _f32(base), _f32(queries)
    n, d = base.shape
    ids = np.empty((queries.shape[0], k), np.int32)
    d2 = np.empty((queries.shape[0], k), np.float64)
    rc = _load().or_knn_queries(_p(base), n, d, _p(queries), queries.shape[0], k, _p(ids), _p(d2))
    if rc != 0:
        raise ValueError("k must be <= n")
    return ids, d2


def pool(base, knn, L, rows=None, own_row_first=False):
    """Candidate pools (Alg. 3) for the given rows.  knn: int32 [n][K] for all nodes.
    own_row_first: the node's whole kNN row first, then its neighbours' rows (the
    alternative reading of the pool loop).
    Returns (ids int32 [m][L] -1 padded, d2 float64 [m][L], len int32 [m])."""
    base, knn = _f32(base), _i32(knn)
    n, d = base.shape
    K = knn.shape[1]
    rows = _i64(np.arange(n) if rows is None else rows)
    ids = np.empty((rows.size, L), np.int32)
    d2 = np.empty((rows.size, L), np.float64)
    ln = np.empty(rows.size, np.int32)
    _load().or_pool2(_p(base), n, d, _p(knn), K, L, _p(rows), rows.size, int(own_row_first),
                     _p(ids), _p(d2), _p(ln))
    return ids, d2, ln


def prune(base, cand, cand_len, R, alpha_deg, nodes=None):
    """SSG prune (Alg. 2 rule) of sorted candidate lists cand [m][stride] for nodes
    (rows 0..m-1 if None).  Returns (adj int32 [m][R] -1 padded, deg int32 [m])."""
    base, cand, cand_len = _f32(base), _i32(cand), _i32(cand_len)
    n, d = base.shape
    m, stride = cand.shape
    nodes = _i64(np.arange(m) if nodes is None else nodes)
    adj = np.empty((m, R), np.int32)
    deg = np.empty(m, np.int32)
    _load().or_prune(_p(base), n, d, _p(nodes), m, _p(cand), _p(cand_len), stride, R,
                     cos_alpha(alpha_deg), _p(adj), _p(deg))
    return adj, deg


def reverse(base, adj0, deg0, alpha_deg):
    """Reverse-neighbour merge (Alg. 3, reading R4).  Returns (adj1, deg1)."""
    base, adj0, deg0 = _f32(base), _i32(adj0), _i32(deg0)
    n, d = base.shape
    R = adj0.shape[1]
    adj1 = np.empty_like(adj0)
    deg1 = np.empty_like(deg0)
    _load().or_reverse(_p(base), n, d, _p(adj0), _p(deg0), R, cos_alpha(alpha_deg),
                       _p(adj1), _p(deg1))
    return adj1, deg1


def connect(base, adj, deg, nav):
    """Connectivity from the navigating nodes (Alg. 3, reading R7).  Works on copies.
    Returns (adj, deg, n_repair); raises RuntimeError if no reached node has a free slot."""
    base = _f32(base)
    adj, deg, nav = _i32(adj).copy(), _i32(deg).copy(), _i32(nav)
    n, d = base.shape
    R = adj.shape[1]
    rep = np.zeros(1, np.int64)
    rc = _load().or_connect(_p(base), n, d, _p(adj), _p(deg), R, _p(nav), nav.size, _p(rep))
    if rc != 0:
        raise RuntimeError("connectivity repair found no reached node with a free slot")
    return adj, deg, int(rep[0])


def search(base, adj, deg, nav, queries, k, Ls):
    """Alg. 1 from the nearest navigating node.  Returns (ids, d2, n_dist, n_hops)."""
    base, adj, deg, nav, queries = _f32(base), _i32(adj), _i32(deg), _i32(nav), _f32(queries)
    n, d = base.shape
    R = adj.shape[1]
    nq = queries.shape[0]
    ids = np.empty((nq, k), np.int32)
    d2 = np.empty((nq, k), np.float64)
    nd = np.empty(nq, np.int64)
    nh = np.empty(nq, np.int64)
    rc = _load().or_search(_p(base), n, d, _p(adj), _p(deg), R, _p(nav), nav.size, _p(queries),
                           nq, k, Ls, _p(ids), _p(d2), _p(nd), _p(nh))
    if rc != 0:
        raise ValueError("need k <= Ls and at least one navigating node")
    return ids, d2, nd, nh


def dist2_pairs(base, a, b):
    base = _f32(base)
    a, b = _i64(a), _i64(b)
    out = np.empty(a.size, np.float64)
    _load().or_dist2_pairs(_p(base), base.shape[1], _p(a), _p(b), a.size, _p(out))
    return out


def cos_triples(base, i, j, k):
    base = _f32(base)
    i, j, k = _i64(i), _i64(j), _i64(k)
    out = np.empty(i.size, np.float64)
    _load().or_cos_triples(_p(base), base.shape[1], _p(i), _p(j), _p(k), i.size, _p(out))
    return out


def recall_at(found_ids, truth_ids, k=10):
    """precision(R) = |R n G| / |G| (Sec. 5.2) averaged over queries, on the first k."""
    f = np.asarray(found_ids)[:, :k]
    g = np.asarray(truth_ids)[:, :k]
    hits = sum(len(set(a.tolist()) & set(b.tolist())) for a, b in zip(f, g))
    return hits / float(g.size)


def build_graph(base, K, L, R, alpha_deg, nav):
    """The whole NSSG build (Alg. 3) through the oracle: kNN -> pool -> prune -> reverse
    -> connect.  Returns a dict of every stage's output."""
    knn_id, knn_d2 = knn_rows(base, K)
    pid, pd2, plen = pool(base, knn_id, L)
    adj0, deg0 = prune(base, pid, plen, R, alpha_deg)
    adj1, deg1 = reverse(base, adj0, deg0, alpha_deg)
    adj, deg, nrep = connect(base, adj1, deg1, nav)
    return dict(knn_id=knn_id, knn_d2=knn_d2, pool_id=pid, pool_d2=pd2, pool_len=plen,
                adj0=adj0, deg0=deg0, adj1=adj1, deg1=deg1, adj=adj, deg=deg, n_repair=nrep,
                nav=np.asarray(nav, np.int32))


def exact_ssg(base, alpha_deg):
    """SSG-Build (Alg. 2): every node's candidates are all other nodes by (d2, id), pruned
    with no degree cap.  For tiny inputs only (O(n^2 log n + n^2 deg d))."""
    base = _f32(base)
    n = base.shape[0]
    ids, _ = knn_rows(base, n - 1)
    return prune(base, ids, np.full(n, n - 1, np.int32), n - 1, alpha_deg)
