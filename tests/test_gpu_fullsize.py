"""Parity at the full size of the benchmark's workload, in the launch configuration bench.py
times: 1,000,000 SIFT-shaped integer vectors (d = 128), K = 200, L = 100, R = 50, alpha =
60, 10 navigating nodes, 10,000 queries.  The oracle cannot build this graph, so it checks
what it can compute one row at a time, and the rest is checked by properties that hold at
any size:

* kNN rows, pools and first prunes of 24 seeded random nodes equal the oracle's exactly
  (integer data: every distance is exact).  The pool of a node reads only its nearest
  neighbour's row here (K >= L: Alg. 3's loop stops after n1), so the oracle needs just
  those rows.
* The reverse merge keeps, for each sampled node, only its pruned edges and in-edges, with
  every pair of kept edges at least alpha apart (exact integer test); and, stage by stage,
  each sampled node's merged row equals the oracle's: its candidates (its edges, then its
  in-edges, from the GPU's first prune) ordered by the oracle's (d2, id) and pruned by the
  oracle's rule.
* After connectivity every node is reachable from each of the navigating nodes, and the
  staged chain equals the one-call build.
* Ground truth of 100 sampled queries equals the oracle's; recall@10 at L_search = 40 over
  all 10,000 queries is at least 0.95.
"""
import numpy as np
import pytest

import oracle
from paper_1907_06146_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K, L, R, ALPHA, N_NAV = 200, 100, 50, 60.0, 10
SAMPLE, QSAMPLE = 24, 100


@pytest.fixture(scope="module")
def ssg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06146_gb300 import build_ext, ssg as S
    build_ext.build()
    S.lib()
    return S


@pytest.fixture(scope="module")
def full(ssg):
    w = synth.sift_like()  # the benchmark's data: 1M x 128, 10,000 queries
    b = torch.from_numpy(w.base).cuda()
    nav = synth.nav_ids(w.n, N_NAV, synth.SEED_DEEP)
    knn_id, knn_d2 = ssg.knn(b, K)
    pid, pd2, pl = ssg.pool(b, knn_id, L)
    adj0, deg0 = ssg.prune(b, pid, pl, R, ALPHA)
    adj1, deg1 = ssg.reverse(b, adj0, deg0, ALPHA)
    adj, deg, nrep = ssg.connect(b, adj1, deg1, nav)
    g = ssg.build(b, K, L, R, ALPHA, nav=nav)
    torch.cuda.synchronize()
    host = {k: v.cpu().numpy() for k, v in dict(knn_id=knn_id, knn_d2=knn_d2, pid=pid, pl=pl,
                                               adj0=adj0, deg0=deg0, adj1=adj1, deg1=deg1,
                                               adj=adj, deg=deg).items()}
    rng = np.random.default_rng(20250)
    sample = np.sort(rng.choice(w.n, SAMPLE, replace=False))
    return w, b, nav, host, nrep, g, sample


def oracle_rows(w, sample):
    """The oracle's kNN rows, pools and first prunes of the sampled nodes."""
    oid, od2 = oracle.knn_rows(w.base, K, rows=sample)
    n1 = oid[:, 0]
    o1, _ = oracle.knn_rows(w.base, K, rows=n1)
    knn = np.zeros((w.n, K), np.int32)  # only the rows the pool loop reads are filled
    knn[sample] = oid
    knn[n1] = o1
    ppid, _, ppl = oracle.pool(w.base, knn, L, rows=sample)
    padj, pdeg = oracle.prune(w.base, ppid, ppl, R, ALPHA, nodes=sample)
    return oid, od2, ppid, ppl, padj, pdeg


def test_sampled_rows_equal_oracle(full):
    w, b, nav, h, nrep, g, sample = full
    oid, od2, ppid, ppl, padj, pdeg = oracle_rows(w, sample)
    np.testing.assert_array_equal(h["knn_id"][sample], oid)
    np.testing.assert_array_equal(h["knn_d2"][sample], od2.astype(np.float32))
    np.testing.assert_array_equal(h["pl"][sample], ppl)
    np.testing.assert_array_equal(h["pid"][sample], ppid)
    np.testing.assert_array_equal(h["deg0"][sample], pdeg)
    np.testing.assert_array_equal(h["adj0"][sample], padj)


def check_reverse(base, adj0, deg0, adj1, deg1, sample):
    """Each sampled node keeps only its own pruned edges and in-edges, once each, and every
    pair of kept edges is at least 60 degrees apart."""
    assert (deg1 >= 0).all() and (deg1 <= adj1.shape[1]).all()
    hit = np.isin(adj0, sample)
    src, col = np.nonzero(hit)
    x = base.astype(np.float64)
    for j in sample:
        kept = adj1[j, :deg1[j]]
        assert (adj1[j, deg1[j]:] == -1).all()
        cand = set(adj0[j, :deg0[j]].tolist()) | set(src[adj0[src, col] == j].tolist())
        assert set(kept.tolist()) <= cand and len(set(kept.tolist())) == len(kept)
        v = x[kept] - x[j]
        gram = v @ v.T
        nn = np.diag(gram)
        for a in range(len(kept)):
            for c in range(a + 1, len(kept)):
                if nn[a] > 0 and nn[c] > 0:
                    # cos > 1/2  <=>  g > 0 and 4 g^2 > |a|^2 |c|^2 (exact on integers)
                    assert not (gram[a, c] > 0 and 4 * gram[a, c] ** 2 > nn[a] * nn[c])


def check_reachable(adj, deg, roots):
    """Degrees within the cap, -1 padding, and every node reachable from each root."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order
    n, cap = adj.shape
    assert (deg >= 1).all() and (deg <= cap).all()
    rows = np.repeat(np.arange(n), deg)
    cols = adj[adj >= 0]  # row-major: each row's first deg entries
    assert rows.size == cols.size
    m = csr_matrix((np.ones(rows.size, np.int8), (rows, cols)), shape=(n, n))
    for root in roots:
        order = breadth_first_order(m, int(root), directed=True, return_predecessors=False)
        assert order.size == n


def test_reverse_merge_properties(full):
    w, b, nav, h, nrep, g, sample = full
    check_reverse(w.base, h["adj0"], h["deg0"], h["adj1"], h["deg1"], sample)


def test_reverse_merge_rows_equal_oracle(full):
    """Reading R4 for the sampled nodes, from the GPU's own first-prune graph: candidates
    adj0[j] then the in-edges {i : j in adj0[i]} (repeats dropped), ordered by the oracle's
    (d2, id), pruned by the oracle with the same cap."""
    w, b, nav, h, nrep, g, sample = full
    adj0, deg0 = h["adj0"], h["deg0"]
    src, col = np.nonzero(np.isin(adj0, sample))
    lists = []
    for j in sample:
        own = adj0[j, :deg0[j]].tolist()
        ins = np.unique(src[adj0[src, col] == j]).tolist()
        cand = np.array(own + [i for i in ins if i not in set(own)], np.int64)
        d2 = oracle.dist2_pairs(w.base, np.full(cand.size, j), cand)
        lists.append(cand[np.lexsort((cand, d2))])
    width = max(len(c) for c in lists)
    cand = np.full((len(sample), width), -1, np.int32)
    clen = np.array([len(c) for c in lists], np.int32)
    for r, c in enumerate(lists):
        cand[r, :len(c)] = c
    oadj, odeg = oracle.prune(w.base, cand, clen, R, ALPHA, nodes=sample)
    np.testing.assert_array_equal(h["deg1"][sample], odeg)
    np.testing.assert_array_equal(h["adj1"][sample], oadj)


def test_connectivity_and_build_equal_staged(full):
    w, b, nav, h, nrep, g, sample = full
    adj, deg = h["adj"], h["deg"]
    check_reachable(adj, deg, nav)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(g.deg.cpu().numpy(), deg)
    np.testing.assert_array_equal(g.adj.cpu().numpy(), adj)
    assert g.stats["n_repair"] == nrep


def test_ground_truth_and_recall(ssg, full):
    w, b, nav, h, nrep, g, sample = full
    q = torch.from_numpy(w.queries).cuda()
    qs = np.arange(0, w.queries.shape[0], w.queries.shape[0] // QSAMPLE)[:QSAMPLE]
    gt_o, gd_o = oracle.knn_queries(w.base, w.queries[qs], 10)
    gt, gd = ssg.knn_query(b, q, 10)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(gt.cpu().numpy()[qs], gt_o)
    np.testing.assert_array_equal(gd.cpu().numpy()[qs], gd_o.astype(np.float32))
    ids, _ = g.search(b, q, 10, 40)
    assert ssg.recall_hits(ids, gt, 10) / (w.queries.shape[0] * 10.0) >= 0.95
