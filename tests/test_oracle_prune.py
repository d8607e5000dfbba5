"""Pins for the oracle's SSG prune (Alg. 2 rule, applied to pools by Alg. 3).

* the hand-derived 3x3 grid (tests/golden/grid3x3_ssg.txt);
* exact integer arithmetic: on integer data the 60/90/120-degree tests reduce to
  comparisons of integers (cos > 1/2 <=> g > 0 and 4 g^2 > g_jj g_kk), evaluated here
  with Python integers;
* the SSG definition of Sec. 3.2 (cone intersected with ball), checked edge by edge with
  angles from arccos;
* Lemma 1 (degree bounded by a function of alpha and d: at most 6 in the plane at 60
  degrees) and the pairwise-angle invariant;
* Theorem 1 (an SSG with alpha <= 60 degrees is an MSNET): a monotonic path exists for
  every ordered pair, and greedy search with l = 1 reaches every indexed query.
"""
import itertools
from collections import deque

import numpy as np
import pytest

import oracle
from paper_1907_06146_gb300 import synth


def _grid():
    pts = [(i % 3 - 1, i // 3 - 1) for i in range(9)]
    return np.array(pts, dtype=np.float32)


def test_grid_golden(golden):
    base = _grid()
    rows = golden("grid3x3_ssg.txt")
    by_alpha = {}
    for head, tail in rows:
        alpha, node = float(head[0]), int(head[1])
        if alpha not in by_alpha:
            by_alpha[alpha] = oracle.exact_ssg(base, alpha)
        adj, deg = by_alpha[alpha]
        want = [int(t) for t in tail.split()]
        assert adj[node, :deg[node]].tolist() == want, (alpha, node)


def _int_conflict(g_jk, g_jj, g_kk, alpha):
    """Exact decision cos > cos(alpha) for integer Gram entries (alpha in 60/90/120)."""
    if g_jj == 0 or g_kk == 0:
        return alpha > 90                 # zero-length edge: its cosine is taken as 0
    if alpha == 60:
        return g_jk > 0 and 4 * g_jk * g_jk > g_jj * g_kk
    if alpha == 90:
        return g_jk > 0
    if alpha == 120:
        return g_jk >= 0 or 4 * g_jk * g_jk < g_jj * g_kk
    raise ValueError(alpha)


def _int_prune(X, i, cand, R, alpha):
    xi = X[i]
    kept = []
    for j in cand:
        if len(kept) == R:
            break
        vj = X[j] - xi
        ok = True
        for k in kept:
            vk = X[k] - xi
            if _int_conflict(int(vj @ vk), int(vj @ vj), int(vk @ vk), alpha):
                ok = False
                break
        if ok:
            kept.append(int(j))
    return kept


@pytest.mark.parametrize("alpha", [60, 90, 120])
def test_prune_integer_exact(alpha):
    base = synth.uniform_points(150, 8, 21, integer=True, hi=15)
    base[10] = base[3]          # a duplicate: a zero-length edge for nodes 3 and 10
    X = base.astype(np.int64)
    ids, _ = oracle.knn_rows(base, 40)
    R = 12
    adj, deg = oracle.prune(base, ids, np.full(150, 40, np.int32), R, alpha)
    for i in range(150):
        assert adj[i, :deg[i]].tolist() == _int_prune(X, i, ids[i], R, alpha), i
        assert np.all(adj[i, deg[i]:] == -1)


def _angle_deg(u, v):
    c = np.dot(u, v) / (np.linalg.norm(u) * np.linalg.norm(v))
    return np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))


@pytest.mark.parametrize("n,d,alpha,seed", [(30, 2, 60, 31), (30, 3, 45, 32), (28, 6, 30, 33),
                                            (30, 2, 20, 34)])
def test_ssg_definition(n, d, alpha, seed):
    """pq in SSG <=> Cone(pq, a) n B(p, |pq|) n S is empty or none of its points r has pr
    in SSG (Sec. 3.2).  Cone: angle(r - p, q - p) < a; ball: open, |pr| < |pq|."""
    base = synth.uniform_points(n, d, seed).astype(np.float64)
    adj, deg = oracle.exact_ssg(base.astype(np.float32), alpha)
    X = base.astype(np.float32).astype(np.float64)
    E = np.zeros((n, n), bool)
    for p in range(n):
        E[p, adj[p, :deg[p]]] = True
    for p in range(n):
        for q in range(n):
            if p == q:
                continue
            dpq = np.sum((X[q] - X[p]) ** 2)
            inside = []
            for r in range(n):
                if r in (p, q):
                    continue
                a = _angle_deg(X[r] - X[p], X[q] - X[p])
                assert abs(a - alpha) > 1e-6          # random data: no boundary cases
                if a < alpha and np.sum((X[r] - X[p]) ** 2) < dpq:
                    inside.append(r)
            expected = len(inside) == 0 or not any(E[p, r] for r in inside)
            assert E[p, q] == expected, (p, q)


def test_degree_bound_plane():
    """Lemma 1: in E^2 with a = 60 degrees, edges pairwise >= 60 degrees apart number <= 6."""
    base = synth.uniform_points(120, 2, 41)
    adj, deg = oracle.exact_ssg(base, 60)
    assert deg.max() <= 6
    assert deg.min() >= 1


@pytest.mark.parametrize("d,alpha", [(2, 60), (5, 60), (5, 45), (16, 75)])
def test_pairwise_angle_invariant(d, alpha):
    base = synth.uniform_points(150, d, 50 + d)
    ids, _ = oracle.knn_rows(base, 60)
    adj, deg = oracle.prune(base, ids, np.full(150, 60, np.int32), 20, alpha)
    X = base.astype(np.float64)
    for i in range(150):
        kept = adj[i, :deg[i]]
        assert kept[0] == ids[i, 0]                # the nearest candidate is always kept
        for a, b in itertools.combinations(kept, 2):
            assert _angle_deg(X[a] - X[i], X[b] - X[i]) >= alpha - 1e-9
        # every rejected candidate before the cap conflicts with a nearer kept edge
        pos = {int(c): t for t, c in enumerate(ids[i])}
        last = pos[int(kept[-1])] if deg[i] == 20 else 60
        for c in ids[i][:last]:
            if c in kept:
                continue
            nearer = [k for k in kept if pos[int(k)] < pos[int(c)]]
            assert any(_angle_deg(X[c] - X[i], X[k] - X[i]) < alpha for k in nearer)


def _monotone_reach(X, E, s, q):
    dq = np.sum((X - X[q]) ** 2, axis=1)
    seen = {s}
    dq_s = deque([s])
    while dq_s:
        u = dq_s.popleft()
        if u == q:
            return True
        for v in np.nonzero(E[u])[0]:
            if v not in seen and dq[v] < dq[u]:
                seen.add(v)
                dq_s.append(v)
    return False


@pytest.mark.parametrize("d,alpha,seed", [(2, 60, 61), (3, 60, 62), (4, 45, 63)])
def test_theorem1_msnet(d, alpha, seed):
    """Theorem 1: with a <= 60 degrees, every ordered pair has a monotonic path."""
    n = 60
    base = synth.uniform_points(n, d, seed)
    adj, deg = oracle.exact_ssg(base, alpha)
    X = base.astype(np.float64)
    E = np.zeros((n, n), bool)
    for p in range(n):
        E[p, adj[p, :deg[p]]] = True
    for s in range(n):
        for q in range(n):
            if s != q:
                assert _monotone_reach(X, E, s, q), (s, q)
    # the search trajectory on an MSNET is monotonic: greedy search with l = 1 started at
    # any node finds any indexed query (the query is a base point, d2 = 0)
    for s in range(0, n, 7):
        ids, d2, _, _ = oracle.search(base, adj, deg, np.array([s]), base, 1, 1)
        np.testing.assert_array_equal(ids[:, 0], np.arange(n))
        assert np.all(d2[:, 0] == 0.0)


def test_cos_alpha_exact_values():
    assert oracle.cos_alpha(60) == 0.5
    assert oracle.cos_alpha(90) == 0.0
    assert oracle.cos_alpha(120) == -0.5
    assert oracle.cos_alpha(45) == pytest.approx(np.sqrt(0.5), rel=1e-15)
