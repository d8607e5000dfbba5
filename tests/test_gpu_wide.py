"""Rows wider than 128 values on the tensor cores: the K-chunked kernel that streams the
query rows with the base tiles (128 x 256 tiles, N = 256 MMAs).  Integer data that bf16
holds exactly (with every distance exact in fp32) give the exact kNN rows directly; float
data (the 960-d GIST-shaped set) go through the certified path.  Every result must equal
the oracle's: kNN ids and distances, ground truth, and a whole build."""
import numpy as np
import pytest

import oracle
from paper_1907_06146_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ssg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_06146_gb300 import build_ext, ssg as S
    build_ext.build()
    S.lib()
    return S


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("n,d,K,hi", [(1100, 130, 10, 100), (2100, 192, 50, 60), (777, 256, 100, 40),
                                      (1500, 960, 30, 10), (300, 4096, 5, 3)])
def test_wide_integer_rows_exact(ssg, n, d, K, hi):
    """Ragged sizes (not multiples of the 128-row or 256-column tiles), one to 64 chunks."""
    base = synth.uniform_points(n, d, 3000 + d, integer=True, hi=hi)
    ids, d2 = ssg.knn(_cuda(base), K, prec="bf16")
    oid, od2 = oracle.knn_rows(base, K)
    np.testing.assert_array_equal(_np(ids), oid)
    np.testing.assert_array_equal(_np(d2), od2.astype(np.float32))


def test_wide_duplicates_settled_by_id(ssg):
    rng = np.random.default_rng(41)
    base = rng.integers(0, 8, size=(900, 200)).astype(np.float32)
    base[rng.choice(900, 300, replace=False)] = base[7]
    ids, d2 = ssg.knn(_cuda(base), 40, prec="bf16")
    oid, od2 = oracle.knn_rows(base, 40)
    np.testing.assert_array_equal(_np(ids), oid)
    np.testing.assert_array_equal(_np(d2), od2.astype(np.float32))


def test_wide_large_self_join(ssg):
    """70,000 rows of 160 values: a self-join large enough that the resident kernel would
    walk the cluster order; the K-chunked kernel walks every row block's columns in the same
    order (for L2 reuse), with many compactions while the thresholds fall."""
    w = synth.sift_like(n=70_000, d=160, nq=0, n_clusters=70)
    base = np.minimum(w.base, 60.0).astype(np.float32)
    ids, d2 = ssg.knn(_cuda(base), 50, prec="bf16")
    ids, d2 = _np(ids), _np(d2)
    rows = np.sort(np.random.default_rng(5).choice(base.shape[0], 150, replace=False))
    oid, od2 = oracle.knn_rows(base, 50, rows=rows)
    np.testing.assert_array_equal(ids[rows], oid)
    np.testing.assert_array_equal(d2[rows], od2.astype(np.float32))


def test_wide_float_certified(ssg):
    w = synth.gist_like(n=2_500, nq=50, n_clusters=10)
    for prec in ("bf16", "auto"):
        ids, d2 = ssg.knn(_cuda(w.base), 40, prec=prec)
        oid, od2 = oracle.knn_rows(w.base, 40)
        np.testing.assert_array_equal(_np(ids), oid)
        np.testing.assert_array_equal(_np(d2), od2.astype(np.float32))
    gi, gd = ssg.knn_query(_cuda(w.base), _cuda(w.queries), 10)
    oi, od = oracle.knn_queries(w.base, w.queries, 10)
    np.testing.assert_array_equal(_np(gi), oi)
    np.testing.assert_array_equal(_np(gd), od.astype(np.float32))


def test_wide_build_equals_oracle(ssg):
    """A GIST-shaped index (960-d, float in [0, 1]): bf16 kNN through the tensor cores,
    certified, then the exact pools, prune, reverse merge and connectivity."""
    w = synth.gist_like(n=1_200, nq=60, n_clusters=8)
    nav = synth.nav_ids(w.n, 4, 61)
    b = _cuda(w.base)
    g = ssg.build(b, 30, 80, 20, 60.0, nav=nav)
    assert g.stats["gemm_prec_used"] == ssg.PREC["bf16"]
    o = oracle.build_graph(w.base, 30, 80, 20, 60.0, nav)
    np.testing.assert_array_equal(_np(g.deg), o["deg"])
    np.testing.assert_array_equal(_np(g.adj), o["adj"])
    g32 = ssg.build(b, 30, 80, 20, 60.0, nav=nav, prec="fp32")
    np.testing.assert_array_equal(_np(g32.adj), o["adj"])


def test_too_wide_rows_refused_for_bf16(ssg):
    base = synth.uniform_points(200, 4100, 3999, integer=True, hi=3)
    ids, d2 = ssg.knn(_cuda(base), 5, prec="auto")
    oid, od2 = oracle.knn_rows(base, 5)
    np.testing.assert_array_equal(_np(ids), oid)
    with pytest.raises(ssg.SSGError):
        ssg.knn(_cuda(base), 5, prec="bf16")


def test_block_prune_spill_and_ties(ssg):
    """The block prune of long rows (d = 960, R = 70).  80 repeated rows give zero-length
    edges and exact distance ties in the pools and the reverse lists.  At 60 degrees a few
    percent of the nodes keep more than 24 vectors, more than the block's shared memory
    holds (the rest live in its device slot); at 35 degrees nearly every node keeps R = 70.  Prune and reverse
    merge at both angles, the pools and the whole build at 60 must equal the oracle."""
    w = synth.gist_like(n=900, nq=0, n_clusters=6)
    base = w.base.copy()
    rng = np.random.default_rng(43)
    base[rng.choice(900, 80, replace=False)] = base[rng.choice(900, 80)]
    nav = synth.nav_ids(900, 3, 67)
    ref = oracle.build_graph(base, 40, 150, 70, 60.0, nav)
    b = _cuda(base)
    pid, _, pl = ssg.pool(b, _cuda(ref["knn_id"]), 150)
    np.testing.assert_array_equal(_np(pl), ref["pool_len"])
    np.testing.assert_array_equal(_np(pid), ref["pool_id"])
    for alpha in (60.0, 35.0):
        if alpha == 60.0:
            a0, d0, a1, d1 = ref["adj0"], ref["deg0"], ref["adj1"], ref["deg1"]
            assert (d0 > 24).mean() > 0.02
        else:
            a0, d0 = oracle.prune(base, ref["pool_id"], ref["pool_len"], 70, alpha)
            a1, d1 = oracle.reverse(base, a0, d0, alpha)[:2]
            assert (d0 == 70).mean() > 0.9
        adj0, deg0 = ssg.prune(b, _cuda(ref["pool_id"]), _cuda(ref["pool_len"]), 70, alpha)
        np.testing.assert_array_equal(_np(deg0), d0)
        np.testing.assert_array_equal(_np(adj0), a0)
        adj1, deg1 = ssg.reverse(b, _cuda(a0), _cuda(d0), alpha)
        np.testing.assert_array_equal(_np(deg1), d1)
        np.testing.assert_array_equal(_np(adj1), a1)
    g = ssg.build(b, 40, 150, 70, 60.0, nav=nav)
    np.testing.assert_array_equal(_np(g.deg), ref["deg"])
    np.testing.assert_array_equal(_np(g.adj), ref["adj"])


def test_block_prune_exact_angles(ssg):
    """0/1 rows of 400 values with four ones among the first 12 columns: many centred
    pairs meet at exactly 60 degrees, where the block prune's fp64 cosine is re-taken in
    coordinate order (an angle of exactly alpha keeps the edge)."""
    rng = np.random.default_rng(44)
    base = np.zeros((600, 400), np.float32)
    for r in range(600):
        base[r, rng.choice(12, 4, replace=False)] = 1.0
    base[:, 12:] = rng.integers(0, 2, size=(600, 388)) * (rng.random((600, 388)) < 0.01)
    knn, _ = oracle.knn_rows(base, 30)
    pool_id, _, pool_len = oracle.pool(base, knn, 100)
    for alpha in (60.0, 45.0):
        a0, d0 = oracle.prune(base, pool_id, pool_len, 70, alpha)
        a1, d1 = oracle.reverse(base, a0, d0, alpha)[:2]
        b = _cuda(base)
        adj0, deg0 = ssg.prune(b, _cuda(pool_id), _cuda(pool_len), 70, alpha)
        np.testing.assert_array_equal(_np(deg0), d0)
        np.testing.assert_array_equal(_np(adj0), a0)
        adj1, deg1 = ssg.reverse(b, _cuda(a0), _cuda(d0), alpha)
        np.testing.assert_array_equal(_np(deg1), d1)
        np.testing.assert_array_equal(_np(adj1), a1)
    # the data do hold pairs at exactly 60 degrees
    x = base[0]
    c = base[pool_id[0, :pool_len[0]]] - x
    g = c @ c.T
    nrm = np.sqrt(np.diag(g))
    with np.errstate(divide="ignore", invalid="ignore"):
        exact = int(np.sum(np.isclose(g / np.outer(nrm, nrm), 0.5, rtol=0, atol=1e-12)))
    assert exact > 0


def _tune(text):
    import os
    import tempfile
    f = tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False)
    f.write(text)
    f.close()
    return f.name


def test_bf16_pairs_forced_equal_oracle(ssg):
    """knn_bf16_pairs = 1: every value goes to the tensor cores as a bf16 pair (hi + lo,
    three products per coordinate); the graph of 960-d and 64-d float rows equals the
    oracle's."""
    import os
    path = _tune("knn_bf16_pairs = 1\n")
    try:
        for w, K, L, R in ((synth.gist_like(n=1_500, nq=0, n_clusters=10), 30, 120, 40),
                           (synth.small(n=3_000, d=64, nq=0, seed=77), 20, 60, 24)):
            nav = synth.nav_ids(w.n, 3, 71)
            g = ssg.build(_cuda(w.base), K, L, R, 60.0, nav=nav, prec="bf16", tune_table=path)
            assert g.stats["knn_bf16_pairs"] == 1
            o = oracle.build_graph(w.base, K, L, R, 60.0, nav)
            np.testing.assert_array_equal(_np(g.deg), o["deg"])
            np.testing.assert_array_equal(_np(g.adj), o["adj"])
    finally:
        os.unlink(path)


def test_bf16_pairs_chosen_where_the_band_is_wide(ssg):
    """200,000 GIST-shaped rows (local intrinsic dimension about 40): a single bf16's band
    holds over a thousand candidates, so the build switches to bf16 pairs by itself; the
    kNN rows of 40 sampled nodes equal the oracle's, and the candidate count stays small."""
    w = synth.gist_like(n=200_000, nq=0)
    b = _cuda(w.base)
    g = ssg.build(b, 100, 300, 70, 60.0, n_nav=4)
    st = g.stats
    assert st["knn_bf16_pairs"] == 1
    assert st["knn_candidates"] < 700
    ids, d2 = ssg.knn(b, 100)
    rows = np.sort(np.random.default_rng(9).choice(w.n, 40, replace=False))
    oid, od2 = oracle.knn_rows(w.base, 100, rows=rows)
    np.testing.assert_array_equal(_np(ids)[rows], oid)
    np.testing.assert_array_equal(_np(d2)[rows], od2.astype(np.float32))
