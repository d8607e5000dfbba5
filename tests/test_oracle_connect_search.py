"""Pins for the oracle's connectivity step (Alg. 3, DFS-spanning from the navigating
nodes; reading: nearest reached node with a free slot links the smallest unreached id)
and Search-on-Graph (Alg. 1, started from the nearest navigating node, Sec. 4.1).

Hand-derived fixtures (tests/golden/connect_search_small.txt), reachability from every
root on random graphs, and the degenerate case of Alg. 1 in which the pool holds the
whole graph, where the result must equal brute force (scipy).
"""
from collections import deque

import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_1907_06146_gb300 import synth

PTS5 = np.array([[0, 0], [1, 0], [0, 1], [10, 0], [11, 0]], dtype=np.float32)
CASES = {
    "A": (3, [[1, 2], [0], [0], [4], [3]]),
    "B": (2, [[1, 2], [0, 2], [0], [4], [3]]),
    "C": (2, [[1, 2], [0, 2], [0, 1], [4], [3]]),
}


def _adj(R, lists):
    adj = np.full((len(lists), R), -1, np.int32)
    deg = np.zeros(len(lists), np.int32)
    for i, l in enumerate(lists):
        adj[i, :len(l)] = l
        deg[i] = len(l)
    return adj, deg


def test_connect_golden(golden):
    for head, tail in golden("connect_search_small.txt"):
        if head[0] != "connect":
            continue
        R, lists = CASES[head[1]]
        nav = np.array([int(t) for t in head[2:]], np.int32)
        adj, deg = _adj(R, lists)
        if tail == "error":
            with pytest.raises(RuntimeError):
                oracle.connect(PTS5, adj, deg, nav)
            continue
        adj2, deg2, nrep = oracle.connect(PTS5, adj, deg, nav)
        added = []
        for v in range(5):
            for u in adj2[v, deg[v]:deg2[v]]:
                added.append((v, int(u)))
        want = [tuple(int(x) for x in e.split("->")) for e in tail.split()]
        assert nrep == len(want)
        assert sorted(added) == sorted(want)


def _reach(adj, deg, s):
    seen = np.zeros(adj.shape[0], bool)
    seen[s] = True
    q = deque([s])
    while q:
        u = q.popleft()
        for v in adj[u, :deg[u]]:
            if not seen[v]:
                seen[v] = True
                q.append(v)
    return seen


def test_connect_random_reaches_all():
    rng = np.random.default_rng(7)
    n, R = 400, 6
    base = synth.uniform_points(n, 3, 71)
    # a sparse random graph with many components
    adj = np.full((n, R), -1, np.int32)
    deg = rng.integers(0, 3, size=n).astype(np.int32)
    for i in range(n):
        adj[i, :deg[i]] = rng.choice(n, size=deg[i], replace=False)
    nav = synth.nav_ids(n, 4, 1234)
    adj2, deg2, nrep = oracle.connect(base, adj, deg, nav)
    assert nrep > 0
    for s in nav:
        assert _reach(adj2, deg2, s).all()
    assert np.all(deg2 <= R)
    # the original edges are untouched; repairs are appended
    for i in range(n):
        np.testing.assert_array_equal(adj2[i, :deg[i]], adj[i, :deg[i]])
    assert int((deg2 - deg).sum()) == nrep


def test_search_golden(golden):
    n = 10
    base = np.arange(n, dtype=np.float32)[:, None]
    lists = [[j for j in (i - 1, i + 1) if 0 <= j < n] for i in range(n)]
    adj, deg = _adj(2, lists)
    q = np.array([[2.2]], dtype=np.float32)
    for head, tail in golden("connect_search_small.txt"):
        if head[0] != "search":
            continue
        Ls, k = int(head[1]), int(head[2])
        ids_s, cnt = tail.split("|")
        ids, d2, nd, nh = oracle.search(base, adj, deg, np.array([9]), q, k, Ls)
        assert ids[0].tolist() == [int(t) for t in ids_s.split()]
        assert [int(nd[0]), int(nh[0])] == [int(t) for t in cnt.split()]


def test_search_full_pool_is_brute_force():
    """With Ls >= n on a graph where every node is reachable from the entry, Alg. 1 visits
    every node, so its first k equal the exact k nearest neighbours."""
    w = synth.small(n=600, nq=30)
    nav = synth.nav_ids(600, 3, 99)
    g = oracle.build_graph(w.base, 10, 40, 12, 60, nav)
    ids, d2, nd, _ = oracle.search(w.base, g["adj"], g["deg"], nav, w.queries, 10, 600)
    D = cdist(w.queries.astype(np.float64), w.base.astype(np.float64), "sqeuclidean")
    for r in range(30):
        order = np.lexsort((np.arange(600), D[r]))
        np.testing.assert_array_equal(ids[r], order[:10])
    assert np.all(nd == 3 + 600 - 1)   # every node's distance once, plus the other navs


def test_search_pads_when_pool_is_short():
    base = np.array([[0.0], [1.0], [2.0]], np.float32)
    adj, deg = _adj(1, [[1], [], []])
    ids, d2, _, _ = oracle.search(base, adj, deg, np.array([0]), np.array([[0.0]], np.float32), 3, 3)
    assert ids[0].tolist() == [0, 1, -1]
    assert np.isinf(d2[0, 2])
