"""Mixed precision on float data (SSG_PREC_BF16): the bf16 tensor cores select candidates
on rows centred before rounding, the candidates are ordered exactly, and each row is
certified against a rigorous bound of the bf16 error (rows that fail take a second
tensor-core pass, then the exact fp32 path).  The result must be the oracle's, bit for bit:
kNN ids and distances, ground truth, and the whole graph; the search over it then gives
the oracle's recall.  Data with many exact ties force every fallback stage."""
import os
import tempfile

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


@pytest.fixture(scope="module")
def fl():
    return synth.small(n=5_000, d=32, nq=200, seed=5151)


def _tune(text):
    f = tempfile.NamedTemporaryFile("w", suffix=".txt", delete=False)
    f.write(text)
    f.close()
    return f.name


@pytest.mark.parametrize("d,n,K", [(32, 5_000, 20), (64, 6_000, 50), (128, 4_000, 100)])
def test_knn_float_exact(ssg, d, n, K):
    w = synth.small(n=n, d=d, nq=0, seed=5152 + d)
    ids, d2 = ssg.knn(_cuda(w.base), K, prec="bf16")
    oid, od2 = oracle.knn_rows(w.base, K)
    np.testing.assert_array_equal(_np(ids), oid)
    np.testing.assert_array_equal(_np(d2), od2.astype(np.float32))


def test_knn_nonnegative_offset_exact(ssg):
    """Values in [0, 1] far from the origin (the GIST-like softplus data): centring before
    rounding keeps the bound tight; the result is exact either way."""
    w = synth.gist_like(n=3_000, d=96, nq=0, n_clusters=12)
    ids, d2 = ssg.knn(_cuda(w.base + 3.0), 30, prec="bf16")
    oid, od2 = oracle.knn_rows(w.base + 3.0, 30)
    np.testing.assert_array_equal(_np(ids), oid)
    np.testing.assert_array_equal(_np(d2), od2.astype(np.float32))


def test_knn_query_float_exact(ssg, fl):
    ids, d2 = ssg.knn_query(_cuda(fl.base), _cuda(fl.queries), 10, prec="bf16")
    oid, od2 = oracle.knn_queries(fl.base, fl.queries, 10)
    np.testing.assert_array_equal(_np(ids), oid)
    np.testing.assert_array_equal(_np(d2), od2.astype(np.float32))


def test_ties_take_every_fallback_stage(ssg):
    """600 copies of one point among 1,400 others: a copy's K nearest are copies at d2 = 0,
    and no bound separates ties, so those rows fail both tensor-core passes and take the
    exact path; ties are settled by id as in the oracle."""
    rng = np.random.default_rng(7)
    base = rng.normal(size=(2_000, 32)).astype(np.float32)
    base[rng.choice(2_000, 600, replace=False)] = base[3]
    ids, d2 = ssg.knn(_cuda(base), 12, prec="bf16")
    oid, od2 = oracle.knn_rows(base, 12)
    np.testing.assert_array_equal(_np(ids), oid)
    np.testing.assert_array_equal(_np(d2), od2.astype(np.float32))


def test_without_sizing_rows_fall_back_exactly(ssg, fl):
    """No sample to size the candidate count (knn_sample_rows = 0): KS = 2K certifies few
    rows, so most take the second pass; the graph is still the oracle's."""
    K, L, R, alpha = 20, 60, 24, 60.0
    nav = synth.nav_ids(fl.n, 3, 53)
    path = _tune("# no sizing sample\nknn_sample_rows = 0\n")
    try:
        g = ssg.build(_cuda(fl.base), K, L, R, alpha, nav=nav, prec="bf16", tune_table=path)
    finally:
        os.unlink(path)
    assert g.stats["knn_candidates"] == 2 * K
    assert g.stats["n_knn_fallback_rows"] > 0
    o = oracle.build_graph(fl.base, K, L, R, alpha, nav)
    np.testing.assert_array_equal(_np(g.deg), o["deg"])
    np.testing.assert_array_equal(_np(g.adj), o["adj"])


def test_knn_integer_exact(ssg):
    w = synth.sift_like(n=3_000, nq=0, n_clusters=30)
    ids, d2 = ssg.knn(_cuda(w.base), 30, prec="bf16")
    oid, od2 = oracle.knn_rows(w.base, 30)
    np.testing.assert_array_equal(_np(ids), oid)
    np.testing.assert_array_equal(_np(d2), od2.astype(np.float32))


def test_build_float_equals_oracle(ssg, fl):
    K, L, R, alpha = 20, 60, 24, 60.0
    nav = synth.nav_ids(fl.n, 3, 53)
    b = _cuda(fl.base)
    g = ssg.build(b, K, L, R, alpha, nav=nav, prec="bf16")
    assert g.stats["gemm_prec_used"] == ssg.PREC["bf16"]
    assert g.stats["knn_candidates"] >= K + 8
    o = oracle.build_graph(fl.base, K, L, R, alpha, nav)
    np.testing.assert_array_equal(_np(g.deg), o["deg"])
    np.testing.assert_array_equal(_np(g.adj), o["adj"])
    truth, _ = oracle.knn_queries(fl.base, fl.queries, 10)
    ids, _ = g.search(b, _cuda(fl.queries), 10, 40)
    oids = oracle.search(fl.base, o["adj"], o["deg"], nav, fl.queries, 10, 40)[0]
    assert abs(oracle.recall_at(_np(ids), truth, 10) - oracle.recall_at(oids, truth, 10)) <= 0.002
    # the plain fp32 path builds the same graph
    g32 = ssg.build(b, K, L, R, alpha, nav=nav, prec="fp32", gram_prec="fp32")
    assert g32.stats["gemm_prec_used"] == ssg.PREC["fp32"]
    np.testing.assert_array_equal(_np(g32.adj), o["adj"])


def test_batch_shaped_index_equals_oracle(ssg):
    """One index shaped like the many-index batch (16-centre mixture, K = 100, R = 32):
    d = 128, L = 200."""
    w = synth.small(n=6_000, d=128, nq=100, seed=5199)
    nav = synth.nav_ids(w.n, 10, 5)
    g = ssg.build(_cuda(w.base), 100, 200, 32, 60.0, nav=nav, prec="bf16")
    assert g.stats["gemm_prec_used"] == ssg.PREC["bf16"]
    o = oracle.build_graph(w.base, 100, 200, 32, 60.0, nav)
    np.testing.assert_array_equal(_np(g.deg), o["deg"])
    np.testing.assert_array_equal(_np(g.adj), o["adj"])


def test_wide_rows_through_the_tensor_cores(ssg):
    # d = 960: the K-chunked tensor-core kernel, certified on these float rows; the plain
    # fp32 path builds the same graph
    w = synth.gist_like(n=600, nq=0, n_clusters=8)
    nav = synth.nav_ids(w.n, 3, 59)
    o = oracle.build_graph(w.base, 10, 30, 12, 60.0, nav)
    for prec, used in (("auto", 1), ("bf16", 1), ("fp32", 0)):
        g = ssg.build(_cuda(w.base), 10, 30, 12, 60.0, nav=nav, prec=prec)
        assert g.stats["gemm_prec_used"] == used
        np.testing.assert_array_equal(_np(g.deg), o["deg"])
        np.testing.assert_array_equal(_np(g.adj), o["adj"])


def test_borderline_count_and_fp8_refused(ssg, fl):
    nav = synth.nav_ids(fl.n, 3, 53)
    b = _cuda(fl.base)
    g0 = ssg.build(b, 20, 60, 24, 60.0, nav=nav, cos_margin=0.0)
    g1 = ssg.build(b, 20, 60, 24, 60.0, nav=nav, cos_margin=0.05)
    # a wider band re-tests (and counts) more decisions in fp64 and changes no edge
    assert g0.stats["n_angle_borderline"] == 0
    assert g1.stats["n_angle_borderline"] > 0
    assert g1.stats["n_angle_fp64"] >= g1.stats["n_angle_borderline"]
    np.testing.assert_array_equal(_np(g0.adj), _np(g1.adj))
    for kw in ({"prec": "fp8"}, {"gram_prec": "fp8"}):
        with pytest.raises(ssg.SSGError) as e:
            ssg.build(b, 20, 60, 24, 60.0, nav=nav, **kw)
        assert e.value.status == 1 and b"FP8" in ssg.lib().ssg_last_error()
