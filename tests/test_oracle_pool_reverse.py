"""Pins for the oracle's candidate pools (Alg. 3, neighbours and neighbours' neighbours
with the break at |P| >= l) and reverse-neighbour merge (Alg. 3, Sec. 4.1).

Hand-derived fixtures (tests/golden/line6_pool_reverse.txt) fix the break rule, the
self-exclusion and the (d2, id) order; set invariants check the same rules on random
data; the reverse merge is checked against its defining properties.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1907_06146_gb300 import synth

LINE = np.array([[0.0], [1.0], [3.0], [6.0], [10.0], [15.0]], dtype=np.float32)
LINE_KNN = np.array([[1, 2], [0, 2], [1, 0], [2, 4], [3, 5], [4, 3]], dtype=np.int32)
LINE_ADJ0 = np.array([[1, -1], [2, -1], [3, -1], [4, -1], [5, -1], [4, 3]], dtype=np.int32)
LINE_DEG0 = np.array([1, 1, 1, 1, 1, 2], dtype=np.int32)


def test_line_knn_is_exact():
    ids, _ = oracle.knn_rows(LINE, 2)
    np.testing.assert_array_equal(ids, LINE_KNN)


def test_pool_golden(golden):
    for head, tail in golden("line6_pool_reverse.txt"):
        if head[0] != "pool":
            continue
        L, node = int(head[1]), int(head[2])
        ids, d2, ln = oracle.pool(LINE, LINE_KNN, L, rows=[node])
        want = [int(t) for t in tail.split()]
        assert ids[0, :ln[0]].tolist() == want, (L, node)
        assert np.all(ids[0, ln[0]:] == -1)


def test_reverse_golden(golden):
    for head, tail in golden("line6_pool_reverse.txt"):
        if head[0] != "reverse":
            continue
        R, node = int(head[1]), int(head[2])
        # the cap is the width of the adjacency rows: cut adj0 to R columns
        adj0 = np.ascontiguousarray(LINE_ADJ0[:, :R])
        deg0 = np.minimum(LINE_DEG0, R)
        adj1, deg1 = oracle.reverse(LINE, adj0, deg0, 60)
        want = [int(t) for t in tail.split()]
        assert adj1[node, :deg1[node]].tolist() == want, (R, node)


@pytest.mark.parametrize("K,L", [(10, 30), (20, 100), (8, 200), (30, 25)])
def test_pool_invariants(K, L):
    w = synth.small(n=1500, nq=1)
    base = w.base
    knn, _ = oracle.knn_rows(base, K)
    ids, d2, ln = oracle.pool(base, knn, L)
    X = base.astype(np.float64)
    for i in range(0, 1500, 37):
        # the collected set: union over knn(i) in order of {n} u knn(n), minus i, stopping
        # after the first n at which it reaches L
        coll = []
        for nb in knn[i]:
            for c in [nb, *knn[nb]]:
                if c != i and c not in coll:
                    coll.append(int(c))
            if len(coll) >= L:
                break
        got = ids[i, :ln[i]]
        assert ln[i] == min(L, len(coll))
        assert len(set(got.tolist())) == ln[i]          # no duplicates
        assert i not in got                              # R1
        assert set(got.tolist()) <= set(coll)            # subset of the 2-hop set
        dd = np.sum((X[got] - X[i]) ** 2, axis=1)
        keys = list(zip(dd, got))
        assert keys == sorted(keys)                      # (d2, id) order
        if len(coll) > L:                                # R2: the L nearest of the set
            rest = sorted(set(coll) - set(got.tolist()))
            drest = np.sum((X[rest] - X[i]) ** 2, axis=1)
            assert drest.min() >= dd.max()
        np.testing.assert_allclose(d2[i, :ln[i]], dd, rtol=1e-12)


def test_reverse_invariants():
    w = synth.small(n=1200, nq=1)
    base = w.base
    knn, _ = oracle.knn_rows(base, 16)
    ids, _, ln = oracle.pool(base, knn, 60)
    R, alpha = 12, 60
    adj0, deg0 = oracle.prune(base, ids, ln, R, alpha)
    adj1, deg1 = oracle.reverse(base, adj0, deg0, alpha)
    X = base.astype(np.float64)
    n = base.shape[0]
    inn = [[] for _ in range(n)]
    for i in range(n):
        for j in adj0[i, :deg0[i]]:
            inn[j].append(i)
    ca = 0.5
    for j in range(n):
        cand = set(adj0[j, :deg0[j]].tolist()) | set(inn[j])
        got = adj1[j, :deg1[j]].tolist()
        assert 1 <= deg1[j] <= R
        assert set(got) <= cand
        assert np.all(adj1[j, deg1[j]:] == -1)
        order = sorted(cand, key=lambda c: (np.sum((X[c] - X[j]) ** 2), c))
        assert got[0] == order[0]
        dd = [np.sum((X[c] - X[j]) ** 2) for c in got]
        assert dd == sorted(dd)
        for a, b in itertools.combinations(got, 2):
            u, v = X[a] - X[j], X[b] - X[j]
            assert np.dot(u, v) / np.sqrt(np.dot(u, u) * np.dot(v, v)) <= ca + 1e-12
        # greedy maximality: every candidate nearer than the last examined one that was
        # dropped conflicts with a kept edge nearer than itself
        stop = order.index(got[-1]) if deg1[j] == R else len(order)
        for c in order[:stop]:
            if c in got:
                continue
            u = X[c] - X[j]
            confl = False
            for k in got:
                if order.index(k) > order.index(c):
                    continue
                v = X[k] - X[j]
                if np.dot(u, v) / np.sqrt(np.dot(u, u) * np.dot(v, v)) > ca:
                    confl = True
            assert confl, (j, c)


# ---- the "own row first" reading of the pool loop ------------------------------------
# Points 0, 1, 3, 6, 10, 15 with K = 2 (LINE_KNN).  Node 3 (x = 6), L = 3: its own row
# {2, 4} enters first; the pool then holds 2 < 3 ids, so the row of node 2 (x = 3) adds
# {1, 0}; by squared distance from 6 that is 2 (9), 4 (16), 1 (25), 0 (36), cut to 3.
# The literal loop instead takes {2} u knn(2) = {2, 1, 0} and stops (3 >= L).
# Node 4 (x = 10), L = 2: own row {3 (16), 5 (25)} already fills the pool; the literal loop
# gives {3} u knn(3) minus 4 = {3, 2}, i.e. 3 (16), 2 (49).
@pytest.mark.parametrize("node,L,own,want", [
    (3, 3, True, [2, 4, 1]), (3, 3, False, [2, 1, 0]),
    (4, 2, True, [3, 5]), (4, 2, False, [3, 2]),
])
def test_pool_own_row_first_line(node, L, own, want):
    ids, d2, ln = oracle.pool(LINE, LINE_KNN, L, rows=[node], own_row_first=own)
    assert ids[0, :ln[0]].tolist() == want


def test_pool_own_row_first_is_the_exact_l_nn_when_k_at_least_l():
    from scipy.spatial.distance import cdist
    w = synth.small(n=400, d=6, nq=0, seed=77)
    K, L = 24, 16
    knn, _ = oracle.knn_rows(w.base, K)
    ids, d2, ln = oracle.pool(w.base, knn, L, own_row_first=True)
    x = w.base.astype(np.float64)
    D = cdist(x, x, "sqeuclidean")
    np.fill_diagonal(D, np.inf)
    for i in range(w.n):
        order = np.lexsort((np.arange(w.n), D[i]))[:L]
        assert ids[i].tolist() == order.tolist()
        assert ln[i] == L


def test_pool_own_row_first_invariants_when_k_below_l():
    w = synth.small(n=500, d=5, nq=0, seed=78)
    K, L = 6, 20
    knn, _ = oracle.knn_rows(w.base, K)
    ids, d2, ln = oracle.pool(w.base, knn, L, own_row_first=True)
    for i in range(w.n):
        p = ids[i, :ln[i]].tolist()
        two_hop = set(knn[i].tolist()) | {int(v) for nb in knn[i] for v in knn[nb]}
        two_hop.discard(i)
        assert len(p) == len(set(p)) and i not in p
        assert set(p) <= two_hop
        assert set(knn[i].tolist()) <= set(p)  # the own row is the nearest K, always kept
        assert ln[i] == min(L, len(two_hop)) or ln[i] == L
        assert np.all(np.diff(d2[i, :ln[i]]) >= 0)
