"""GPU parity: every stage of the CUDA path against the CPU oracle, element by element.

Stages are isolated: each GPU stage takes the oracle's output of the previous stage as
its input (oracle -> GPU only; no oracle input ever comes from the GPU).  The bar:
adjacency, pools and kNN ids bit-exact (the library re-decides every near-boundary case
in double precision); search recall@10 within 0.002 of the oracle's on float data and
ids identical on integer data, where every distance is exact in single precision.
Sizes span several 128-row tiles with a ragged tail.
"""
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
def small():
    return synth.small(n=4_000, nq=300)


@pytest.fixture(scope="module")
def intdata():
    return synth.sift_like(n=6_000, nq=300, n_clusters=40)


@pytest.fixture(scope="module")
def small_ref(small):
    nav = synth.nav_ids(small.n, small.n_nav, 11)
    return oracle.build_graph(small.base, small.K, small.L, small.R, small.alpha, nav)


@pytest.fixture(scope="module")
def int_ref(intdata):
    nav = synth.nav_ids(intdata.n, intdata.n_nav, 12)
    return oracle.build_graph(intdata.base, intdata.K, intdata.L, intdata.R, intdata.alpha, nav)


# ---- a1: exact kNN graph ---------------------------------------------------------------
def test_knn_small_float(ssg, small, small_ref):
    ids, d2 = ssg.knn(_cuda(small.base), small.K)
    np.testing.assert_array_equal(_np(ids), small_ref["knn_id"])
    np.testing.assert_array_equal(_np(d2), small_ref["knn_d2"].astype(np.float32))


def test_knn_integer_exact(ssg, intdata, int_ref):
    for prec in ("fp32", "auto"):
        ids, d2 = ssg.knn(_cuda(intdata.base), intdata.K, prec=prec)
        np.testing.assert_array_equal(_np(ids), int_ref["knn_id"])
        np.testing.assert_array_equal(_np(d2), int_ref["knn_d2"].astype(np.float32))


def _tc(ssg):
    return ssg.lib() is not None and _has_tc(ssg)


def _has_tc(ssg):
    # the bf16 path is taken only on sm_103 with exact (small-integer) data
    base = np.arange(64 * 8, dtype=np.float32).reshape(64, 8) % 7
    try:
        ssg.knn(_cuda(base), 3, prec="bf16")
        return True
    except ssg.SSGError:
        return False


@pytest.mark.parametrize("n,d,K", [(1037, 7, 1), (1037, 7, 20), (3001, 64, 200), (900, 96, 600),
                                   (6000, 128, 200)])
def test_knn_bf16_tensor_cores(ssg, n, d, K):
    if not _tc(ssg):
        pytest.skip("bf16 tensor-core kNN needs sm_103")
    base = synth.uniform_points(n, d, 2000 + d, integer=True, hi=255 if d <= 128 else 100)
    ids, d2 = ssg.knn(_cuda(base), K, prec="bf16")
    ref_ids, ref_d2 = oracle.knn_rows(base, K)
    np.testing.assert_array_equal(_np(ids), ref_ids)
    np.testing.assert_array_equal(_np(d2), ref_d2.astype(np.float32))


def test_knn_bf16_near_first_order(ssg):
    """Self-joins of at least 65536 rows with K >= 16 visit the columns cluster by cluster,
    nearest clusters first.  Sampled rows against the oracle (self dropped from its K+1
    nearest), and every row sorted by (d2, id) with distinct ids and no self."""
    if not _tc(ssg):
        pytest.skip("bf16 tensor-core kNN needs sm_103")
    w = synth.sift_like(n=70_001, nq=10)
    K = 200
    ids, d2 = ssg.knn(_cuda(w.base), K, prec="bf16")
    ids, d2 = _np(ids), _np(d2)
    rng = np.random.default_rng(5)
    rows = np.sort(rng.choice(w.n, 160, replace=False))
    rows[-1] = w.n - 1
    ref_ids, ref_d2 = oracle.knn_queries(w.base, w.base[rows], K + 1)
    for i, r in enumerate(rows):
        keep = ref_ids[i] != r
        np.testing.assert_array_equal(ids[r], ref_ids[i][keep][:K])
        np.testing.assert_array_equal(d2[r], ref_d2[i][keep][:K].astype(np.float32))
    assert (ids >= 0).all() and (ids < w.n).all()
    assert not (ids == np.arange(w.n)[:, None]).any()
    srt = np.sort(ids, axis=1)
    assert not (srt[:, 1:] == srt[:, :-1]).any()
    order_ok = (d2[:, 1:] > d2[:, :-1]) | ((d2[:, 1:] == d2[:, :-1]) & (ids[:, 1:] > ids[:, :-1]))
    assert order_ok.all()
    sel = rng.choice(w.n, 500, replace=False)
    x = w.base[sel].astype(np.float64)
    y = w.base[ids[sel]].astype(np.float64)
    np.testing.assert_array_equal(d2[sel], ((x[:, None, :] - y) ** 2).sum(-1).astype(np.float32))


def test_knn_bf16_near_first_order_duplicates(ssg):
    """Cluster order with 401 copies of one point: ties at distance 0 outnumber the
    buffer's room, so the compaction falls back to a sort by (distance, original id)."""
    if not _tc(ssg):
        pytest.skip("bf16 tensor-core kNN needs sm_103")
    w = synth.sift_like(n=66_000, nq=10)
    base = w.base.copy()
    base[1000:1400] = base[5]
    K = 200
    ids, d2 = ssg.knn(_cuda(base), K, prec="bf16")
    ids, d2 = _np(ids), _np(d2)
    rows = np.array([5, 1000, 1200, 1399, 7, 65_999])
    ref_ids, ref_d2 = oracle.knn_queries(base, base[rows], K + 1)
    for i, r in enumerate(rows):
        keep = ref_ids[i] != r
        np.testing.assert_array_equal(ids[r], ref_ids[i][keep][:K])
        np.testing.assert_array_equal(d2[r], ref_d2[i][keep][:K].astype(np.float32))


def test_knn_bf16_signed_integers(ssg):
    """Negative values: the exact tensor-core GEMM needs 4 d max|x|^2 <= 2^24 (squared
    distances up to 4 d max|x|^2 must stay exact); within it bf16 is exact by itself, beyond
    it bf16 values are not exact and the certified path (bounded error, exact re-rank) runs,
    with the same result as the fp32 path and the oracle."""
    if not _tc(ssg):
        pytest.skip("bf16 tensor-core kNN needs sm_103")
    rng = np.random.default_rng(31)
    inside = rng.integers(-100, 101, size=(2100, 64)).astype(np.float32)   # 4*64*100^2 < 2^24
    ids, d2 = ssg.knn(_cuda(inside), 30, prec="bf16")
    ref_ids, ref_d2 = oracle.knn_rows(inside, 30)
    np.testing.assert_array_equal(_np(ids), ref_ids)
    np.testing.assert_array_equal(_np(d2), ref_d2.astype(np.float32))
    beyond = rng.integers(-200, 201, size=(1500, 128)).astype(np.float32)  # 4*128*200^2 > 2^24
    ids, d2 = ssg.knn(_cuda(beyond), 30, prec="auto")
    ref_ids, ref_d2 = oracle.knn_rows(beyond, 30)
    np.testing.assert_array_equal(_np(ids), ref_ids)
    np.testing.assert_array_equal(_np(d2), ref_d2.astype(np.float32))
    ids, d2 = ssg.knn(_cuda(beyond), 30, prec="bf16")
    np.testing.assert_array_equal(_np(ids), ref_ids)
    np.testing.assert_array_equal(_np(d2), ref_d2.astype(np.float32))
    ids, d2 = ssg.knn(_cuda(beyond), 30, prec="fp32")
    np.testing.assert_array_equal(_np(ids), ref_ids)


def test_knn_wide_integer_rows(ssg):
    """d > 128 streams through the K-chunked tensor-core kernel (exact on these integers);
    the fp32 path gives the same rows."""
    base = synth.uniform_points(700, 130, 2130, integer=True, hi=100)
    ref_ids, ref_d2 = oracle.knn_rows(base, 50)
    for prec in ("auto", "bf16", "fp32"):
        ids, d2 = ssg.knn(_cuda(base), 50, prec=prec)
        np.testing.assert_array_equal(_np(ids), ref_ids)
        np.testing.assert_array_equal(_np(d2), ref_d2.astype(np.float32))


def test_ground_truth_bf16(ssg, intdata):
    if not _tc(ssg):
        pytest.skip("bf16 tensor-core kNN needs sm_103")
    ids, d2 = ssg.knn_query(_cuda(intdata.base), _cuda(intdata.queries), 10, prec="bf16")
    ref_ids, ref_d2 = oracle.knn_queries(intdata.base, intdata.queries, 10)
    np.testing.assert_array_equal(_np(ids), ref_ids)
    np.testing.assert_array_equal(_np(d2), ref_d2.astype(np.float32))


@pytest.mark.parametrize("n,d,K", [(1037, 3, 1), (1037, 3, 7), (1300, 33, 200), (700, 17, 640)])
def test_knn_ragged(ssg, n, d, K):
    base = synth.uniform_points(n, d, 1000 + d)
    ids, d2 = ssg.knn(_cuda(base), K)
    ref_ids, ref_d2 = oracle.knn_rows(base, K)
    np.testing.assert_array_equal(_np(ids), ref_ids)
    np.testing.assert_array_equal(_np(d2), ref_d2.astype(np.float32))


def test_knn_duplicates(ssg):
    base = synth.uniform_points(900, 8, 77)
    base[100:130] = base[5]          # 31 copies of one point
    base[500] = base[501]
    ids, d2 = ssg.knn(_cuda(base), 40)
    ref_ids, ref_d2 = oracle.knn_rows(base, 40)
    np.testing.assert_array_equal(_np(ids), ref_ids)
    np.testing.assert_array_equal(_np(d2), ref_d2.astype(np.float32))


def test_ground_truth_queries(ssg, small, intdata):
    for w in (small, intdata):
        ids, d2 = ssg.knn_query(_cuda(w.base), _cuda(w.queries), 10)
        ref_ids, ref_d2 = oracle.knn_queries(w.base, w.queries, 10)
        np.testing.assert_array_equal(_np(ids), ref_ids)
        np.testing.assert_array_equal(_np(d2), ref_d2.astype(np.float32))


# ---- a2: candidate pools -----------------------------------------------------------------
@pytest.mark.parametrize("which", ["small", "int"])
def test_pool(ssg, which, small, intdata, small_ref, int_ref):
    w, ref = (small, small_ref) if which == "small" else (intdata, int_ref)
    pid, pd2, pl = ssg.pool(_cuda(w.base), _cuda(ref["knn_id"]), w.L)
    np.testing.assert_array_equal(_np(pl), ref["pool_len"])
    np.testing.assert_array_equal(_np(pid), ref["pool_id"])


def test_pool_small_L(ssg, small):
    knn, _ = oracle.knn_rows(small.base, 10)
    ref = oracle.pool(small.base, knn, 30)
    pid, _, pl = ssg.pool(_cuda(small.base), _cuda(knn), 30)
    np.testing.assert_array_equal(_np(pl), ref[2])
    np.testing.assert_array_equal(_np(pid), ref[0])


# ---- a3: SSG prune -----------------------------------------------------------------------
@pytest.mark.parametrize("which", ["small", "int"])
def test_prune(ssg, which, small, intdata, small_ref, int_ref):
    w, ref = (small, small_ref) if which == "small" else (intdata, int_ref)
    adj, deg = ssg.prune(_cuda(w.base), _cuda(ref["pool_id"]), _cuda(ref["pool_len"]), w.R, w.alpha)
    np.testing.assert_array_equal(_np(deg), ref["deg0"])
    np.testing.assert_array_equal(_np(adj), ref["adj0"])


@pytest.mark.parametrize("alpha,R", [(45.0, 32), (90.0, 8), (30.0, 64), (75.0, 5)])
def test_prune_angles(ssg, small, small_ref, alpha, R):
    ref = oracle.prune(small.base, small_ref["pool_id"], small_ref["pool_len"], R, alpha)
    adj, deg = ssg.prune(_cuda(small.base), _cuda(small_ref["pool_id"]),
                         _cuda(small_ref["pool_len"]), R, alpha)
    np.testing.assert_array_equal(_np(deg), ref[1])
    np.testing.assert_array_equal(_np(adj), ref[0])


@pytest.mark.parametrize("alpha,R", [(60.0, 50), (30.0, 128), (90.0, 7), (120.0, 20), (150.0, 1)])
def test_prune_integer_angles(ssg, intdata, int_ref, alpha, R):
    """Integer data take the tensor-core Gram prune (exact centred Gram from one UMMA)."""
    ref = oracle.prune(intdata.base, int_ref["pool_id"], int_ref["pool_len"], R, alpha)
    adj, deg = ssg.prune(_cuda(intdata.base), _cuda(int_ref["pool_id"]),
                         _cuda(int_ref["pool_len"]), R, alpha)
    np.testing.assert_array_equal(_np(deg), ref[1])
    np.testing.assert_array_equal(_np(adj), ref[0])


def test_prune_integer_duplicates_full_tile(ssg):
    """d = 7 (one K-chunk), pools of the tile's limit (L = 127) and duplicate points, so
    zero-length edges occur; alpha above 90 degrees makes them conflicts."""
    base = synth.uniform_points(1500, 7, 77, integer=True, hi=6)
    base[100:140] = base[3]
    knn, _ = oracle.knn_rows(base, 40)
    pid, _, pl = oracle.pool(base, knn, 127)
    for alpha in (60.0, 120.0):
        ref = oracle.prune(base, pid, pl, 32, alpha)
        adj, deg = ssg.prune(_cuda(base), _cuda(pid), _cuda(pl), 32, alpha)
        np.testing.assert_array_equal(_np(deg), ref[1])
        np.testing.assert_array_equal(_np(adj), ref[0])


def test_prune_tensor_core_exact_angles_ragged_pools(ssg):
    """0/1 rows of 64 values with four ones among the first 12 columns: many centred pairs
    meet at exactly 60 degrees, where the tensor-core prune's fp64 re-test decides (an
    angle of exactly alpha keeps the edge), both against the candidates kept in earlier
    blocks of 32 and among a block's survivors.  Pool lengths are cut at random (0 to 127
    candidates), so that empty pools and every block boundary occur; repeated rows give
    zero-length edges (conflicts above 90 degrees); R = 3 stops inside the first block."""
    rng = np.random.default_rng(45)
    n, d = 3000, 64
    base = np.zeros((n, d), np.float32)
    for r in range(n):
        base[r, rng.choice(12, 4, replace=False)] = 1.0
    base[:, 12:] = (rng.random((n, d - 12)) < 0.02).astype(np.float32)
    knn, _ = oracle.knn_rows(base, 60)
    pid, _, pl = oracle.pool(base, knn, 127)
    pl = np.minimum(pl, rng.integers(0, 128, size=n)).astype(np.int32)
    pid = np.where(np.arange(127)[None, :] < pl[:, None], pid, -1).astype(np.int32)
    assert (pl == 0).any() and (pl == 127).any()
    for alpha, R in ((60.0, 70), (60.0, 3), (45.0, 128), (100.0, 20)):
        ref = oracle.prune(base, pid, pl, R, alpha)
        adj, deg = ssg.prune(_cuda(base), _cuda(pid), _cuda(pl), R, alpha)
        np.testing.assert_array_equal(_np(deg), ref[1])
        np.testing.assert_array_equal(_np(adj), ref[0])
    # the data do hold centred pairs at exactly 60 degrees
    i = int(np.argmax(pl))
    c = base[pid[i, :pl[i]]] - base[i]
    g = c.astype(np.float64) @ c.T.astype(np.float64)
    nrm = np.sqrt(np.diag(g))
    with np.errstate(divide="ignore", invalid="ignore"):
        assert int(np.sum(np.isclose(g / np.outer(nrm, nrm), 0.5, rtol=0, atol=1e-12))) > 0


# ---- a4: reverse merge -------------------------------------------------------------------
@pytest.mark.parametrize("which", ["small", "int"])
def test_reverse(ssg, which, small, intdata, small_ref, int_ref):
    w, ref = (small, small_ref) if which == "small" else (intdata, int_ref)
    adj1, deg1 = ssg.reverse(_cuda(w.base), _cuda(ref["adj0"]), _cuda(ref["deg0"]), w.alpha)
    np.testing.assert_array_equal(_np(deg1), ref["deg1"])
    np.testing.assert_array_equal(_np(adj1), ref["adj1"])


def test_reverse_hub(ssg):
    """A node that every other node points at: its in-degree exceeds the per-warp buffer."""
    n, R = 1200, 6
    base = synth.uniform_points(n, 5, 91)
    rng = np.random.default_rng(3)
    adj0 = np.full((n, R), -1, np.int32)
    deg0 = np.zeros(n, np.int32)
    for i in range(n):
        others = rng.choice(n, size=4, replace=False)
        row = [0] + [int(x) for x in others if x not in (0, i)]
        row = [x for x in row if x != i][:R]
        adj0[i, :len(row)] = row
        deg0[i] = len(row)
    ref = oracle.reverse(base, adj0, deg0, 60.0)
    adj1, deg1 = ssg.reverse(_cuda(base), _cuda(adj0), _cuda(deg0), 60.0)
    np.testing.assert_array_equal(_np(deg1), ref[1])
    np.testing.assert_array_equal(_np(adj1), ref[0])


@pytest.mark.parametrize("alpha", [60.0, 120.0])
def test_reverse_hub_integer(ssg, alpha):
    """Integer data: lists of up to 127 candidates are pruned on the tensor cores, the hub's
    (over a thousand) by the warp path; duplicates give zero-length edges."""
    n, R = 1200, 6
    base = synth.uniform_points(n, 5, 92, integer=True, hi=40)
    base[50:60] = base[7]
    rng = np.random.default_rng(4)
    adj0 = np.full((n, R), -1, np.int32)
    deg0 = np.zeros(n, np.int32)
    for i in range(n):
        others = rng.choice(n, size=4, replace=False)
        row = [0] + [int(x) for x in others if x not in (0, i)]
        row = [x for x in row if x != i][:R]
        adj0[i, :len(row)] = row
        deg0[i] = len(row)
    ref = oracle.reverse(base, adj0, deg0, alpha)
    adj1, deg1 = ssg.reverse(_cuda(base), _cuda(adj0), _cuda(deg0), alpha)
    np.testing.assert_array_equal(_np(deg1), ref[1])
    np.testing.assert_array_equal(_np(adj1), ref[0])


# ---- a5: connectivity --------------------------------------------------------------------
@pytest.mark.parametrize("which", ["small", "int"])
def test_connect(ssg, which, small, intdata, small_ref, int_ref):
    w, ref = (small, small_ref) if which == "small" else (intdata, int_ref)
    adj, deg, nrep = ssg.connect(_cuda(w.base), _cuda(ref["adj1"]), _cuda(ref["deg1"]),
                                 _cuda(ref["nav"]))
    assert nrep == ref["n_repair"]
    np.testing.assert_array_equal(_np(deg), ref["deg"])
    np.testing.assert_array_equal(_np(adj), ref["adj"])


def test_connect_many_components(ssg):
    rng = np.random.default_rng(7)
    n, R = 3000, 6
    base = synth.uniform_points(n, 3, 71)
    adj = np.full((n, R), -1, np.int32)
    deg = rng.integers(0, 3, size=n).astype(np.int32)
    for i in range(n):
        adj[i, :deg[i]] = rng.choice(n, size=deg[i], replace=False)
    nav = synth.nav_ids(n, 4, 1234)
    ref = oracle.connect(base, adj, deg, nav)
    a, dg, nrep = ssg.connect(_cuda(base), _cuda(adj), _cuda(deg), _cuda(nav))
    assert nrep == ref[2] and nrep > 100
    np.testing.assert_array_equal(_np(dg), ref[1])
    np.testing.assert_array_equal(_np(a), ref[0])


def test_build_repairs_by_knn_row_and_by_scan(ssg):
    """60 tight clusters far apart, K = 8: no kNN row leaves its cluster, so the first
    repair into a cluster finds no reached node in the unreached node's row and scans all
    nodes, while repairs inside a reached cluster are settled from the row.  Both routes
    must give the oracle's graph."""
    rng = np.random.default_rng(77)
    centres = rng.normal(size=(60, 8)) * 100.0
    lab = rng.integers(0, 60, size=2400)
    base = (centres[lab] + rng.normal(size=(2400, 8))).astype(np.float32)
    nav = synth.nav_ids(2400, 3, 17)
    ref = oracle.build_graph(base, 8, 16, 6, 60.0, nav)
    g = ssg.build(_cuda(base), 8, 16, 6, 60.0, nav=nav)
    np.testing.assert_array_equal(_np(g.deg), ref["deg"])
    np.testing.assert_array_equal(_np(g.adj), ref["adj"])
    st = g.stats
    assert st["n_repair"] == ref["n_repair"]
    # replay the repairs on the host: which of them had a qualifying node in u's row
    knn, _ = oracle.knn_rows(base, 8)
    adj, deg, n = ref["adj1"].copy(), ref["deg1"].copy(), base.shape[0]
    by_row = 0
    for s in nav:
        reached = _reach(adj, deg, s, np.zeros(n, bool))
        while not reached.all():
            u = int(np.argmin(reached))
            row = [v for v in knn[u] if reached[v] and deg[v] < 6]
            by_row += bool(row)
            if row:
                v = row[0]
            else:
                ok = np.flatnonzero(reached & (deg < 6))
                d2 = ((base[ok].astype(np.float64) - base[u]) ** 2).sum(1)
                v = int(ok[np.lexsort((ok, d2))[0]])
            adj[v, deg[v]] = u
            deg[v] += 1
            reached = _reach(adj, deg, u, reached)
    np.testing.assert_array_equal(adj, ref["adj"])
    assert st["n_repair_knn_row"] == by_row
    assert 0 < by_row and st["n_repair"] - by_row >= 59


def _reach(adj, deg, s, reached):
    stack = [s]
    reached[s] = True
    while stack:
        x = stack.pop()
        for y in adj[x, :deg[x]]:
            if not reached[y]:
                reached[y] = True
                stack.append(y)
    return reached


# ---- whole build ---------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["small", "int"])
def test_build_end_to_end(ssg, which, small, intdata, small_ref, int_ref):
    w, ref = (small, small_ref) if which == "small" else (intdata, int_ref)
    g = ssg.build(_cuda(w.base), w.K, w.L, w.R, w.alpha, nav=ref["nav"])
    np.testing.assert_array_equal(_np(g.nav), ref["nav"])
    np.testing.assert_array_equal(_np(g.deg), ref["deg"])
    np.testing.assert_array_equal(_np(g.adj), ref["adj"])
    st = g.stats
    assert st["n_repair"] == ref["n_repair"]
    assert st["kernel_launches"] > 5
    assert st["exact_mode"] == (1 if which == "int" else 0)


@pytest.fixture(scope="module")
def wide():
    """GIST-shaped rows (d = 960, values in [0, 1]) at a size the oracle builds quickly;
    R = 70 rows of 960 floats do not fit in shared memory, so the prune and the reverse
    merge take their wide-row path."""
    w = synth.gist_like(n=1_200, nq=60, n_clusters=12)
    nav = synth.nav_ids(w.n, w.n_nav, 13)
    ref = oracle.build_graph(w.base, 50, 200, 70, 60.0, nav)
    return w, ref


def test_wide_rows_prune_reverse_build(ssg, wide):
    w, ref = wide
    b = _cuda(w.base)
    adj0, deg0 = ssg.prune(b, _cuda(ref["pool_id"]), _cuda(ref["pool_len"]), 70, 60.0)
    np.testing.assert_array_equal(_np(deg0), ref["deg0"])
    np.testing.assert_array_equal(_np(adj0), ref["adj0"])
    adj1, deg1 = ssg.reverse(b, _cuda(ref["adj0"]), _cuda(ref["deg0"]), 60.0)
    np.testing.assert_array_equal(_np(deg1), ref["deg1"])
    np.testing.assert_array_equal(_np(adj1), ref["adj1"])
    g = ssg.build(b, 50, 200, 70, 60.0, nav=ref["nav"])
    np.testing.assert_array_equal(_np(g.deg), ref["deg"])
    np.testing.assert_array_equal(_np(g.adj), ref["adj"])


def test_build_host_matches_device(ssg, small, small_ref):
    g, adj, deg = ssg.build_host(small.base, small.K, small.L, small.R, small.alpha,
                                 nav=small_ref["nav"])
    np.testing.assert_array_equal(deg, small_ref["deg"])
    np.testing.assert_array_equal(adj, small_ref["adj"])
    ids, _ = g.search_host(small.queries, 10, 40)
    oid, _, _, _ = oracle.search(small.base, small_ref["adj"], small_ref["deg"], small_ref["nav"],
                                 small.queries, 10, 40)
    truth, _ = oracle.knn_queries(small.base, small.queries, 10)
    assert abs(oracle.recall_at(ids, truth) - oracle.recall_at(oid, truth)) <= 0.002


def test_save_load(ssg, small, small_ref, tmp_path):
    g = ssg.build(_cuda(small.base), small.K, small.L, small.R, small.alpha, nav=small_ref["nav"])
    p = str(tmp_path / "g.nssg")
    g.save(p)
    h = ssg.Graph.load(p)
    np.testing.assert_array_equal(_np(h.adj), small_ref["adj"])
    np.testing.assert_array_equal(_np(h.nav), small_ref["nav"])


# ---- a6 / a7: search and recall -----------------------------------------------------------
@pytest.mark.parametrize("Ls", [10, 20, 40, 80])
def test_search_float_recall(ssg, small, small_ref, Ls):
    ids, _ = ssg.search_adj(_cuda(small.base), _cuda(small_ref["adj"]), _cuda(small_ref["deg"]),
                            _cuda(small_ref["nav"]), _cuda(small.queries), 10, Ls)
    oid, _, _, _ = oracle.search(small.base, small_ref["adj"], small_ref["deg"], small_ref["nav"],
                                 small.queries, 10, Ls)
    truth, _ = oracle.knn_queries(small.base, small.queries, 10)
    g_ids = _np(ids)
    assert abs(oracle.recall_at(g_ids, truth) - oracle.recall_at(oid, truth)) <= 0.002
    assert np.mean(np.all(g_ids == oid, axis=1)) > 0.97


@pytest.mark.parametrize("Ls", [10, 50, 200])
def test_search_integer_exact(ssg, intdata, int_ref, Ls):
    ids, d2 = ssg.search_adj(_cuda(intdata.base), _cuda(int_ref["adj"]), _cuda(int_ref["deg"]),
                             _cuda(int_ref["nav"]), _cuda(intdata.queries), 10, Ls)
    oid, od2, _, _ = oracle.search(intdata.base, int_ref["adj"], int_ref["deg"], int_ref["nav"],
                                   intdata.queries, 10, Ls)
    np.testing.assert_array_equal(_np(ids), oid)
    np.testing.assert_array_equal(_np(d2), od2.astype(np.float32))


def test_search_full_pool_is_brute_force(ssg):
    w = synth.small(n=900, nq=50)
    nav = synth.nav_ids(900, 3, 5)
    ref = oracle.build_graph(w.base, 10, 40, 12, 60, nav)
    ids, _ = ssg.search_adj(_cuda(w.base), _cuda(ref["adj"]), _cuda(ref["deg"]), _cuda(nav),
                            _cuda(w.queries), 10, 1024)
    truth, _ = oracle.knn_queries(w.base, w.queries, 10)
    np.testing.assert_array_equal(_np(ids), truth)


def test_recall_hits(ssg, small):
    truth, _ = oracle.knn_queries(small.base, small.queries, 10)
    found = truth.copy()
    found[::2, 3] = -1
    found[1::3, 0] = 10**6
    hits = ssg.recall_hits(_cuda(found), _cuda(truth), 10)
    assert hits / truth.size == pytest.approx(oracle.recall_at(found, truth))


# ---- the own-row-first pool reading through the whole build ---------------------------
@pytest.mark.parametrize("which", ["small", "intdata"])
def test_build_own_row_first_equals_oracle(ssg, request, which):
    # small: K = 20 < L = 100, so neighbours' rows follow the own row; intdata: K = 200 >= L,
    # so the pool is the node's own 100 nearest
    w = request.getfixturevalue(which)
    nav = synth.nav_ids(w.n, w.n_nav, 61)
    g = ssg.build(_cuda(w.base), w.K, w.L, w.R, w.alpha, nav=nav, pool_own_row_first=True)
    knn, _ = oracle.knn_rows(w.base, w.K)
    pid, _, plen = oracle.pool(w.base, knn, w.L, own_row_first=True)
    adj0, deg0 = oracle.prune(w.base, pid, plen, w.R, w.alpha)
    adj1, deg1 = oracle.reverse(w.base, adj0, deg0, w.alpha)
    adj, deg, _ = oracle.connect(w.base, adj1, deg1, nav)
    np.testing.assert_array_equal(_np(g.deg), deg)
    np.testing.assert_array_equal(_np(g.adj), adj)
