"""Search over the byte copy of integer rows (0..255).

A graph built from data that are integers 0..255 keeps a byte copy of the rows, and its
searches read that copy instead of the float rows.  The values are the same and each lane
sums them in the same order, so the results must be bit for bit those of the float rows --
for integer queries and for arbitrary float queries -- and, on integer data, the oracle's.
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


@pytest.fixture(scope="module", params=[128, 45])
def built(request, ssg):
    d = request.param
    w = synth.sift_like(n=5_000, d=d, nq=300, n_clusters=40)
    nav = synth.nav_ids(w.n, w.n_nav, 17)
    ref = oracle.build_graph(w.base, w.K, w.L, w.R, w.alpha, nav)
    base = _cuda(w.base)
    g = ssg.build(base, w.K, w.L, w.R, w.alpha, nav=nav)
    return w, ref, base, g


def test_graph_equals_oracle(built):
    w, ref, base, g = built
    np.testing.assert_array_equal(_np(g.deg), ref["deg"])
    np.testing.assert_array_equal(_np(g.adj), ref["adj"])


@pytest.mark.parametrize("Ls", [10, 64, 300])
def test_byte_rows_integer_queries_equal_oracle(ssg, built, Ls):
    w, ref, base, g = built
    ids, d2 = g.search(base, _cuda(w.queries), 10, Ls)
    oid, od2, _, _ = oracle.search(w.base, ref["adj"], ref["deg"], ref["nav"], w.queries, 10, Ls)
    np.testing.assert_array_equal(_np(ids), oid)
    np.testing.assert_array_equal(_np(d2), od2.astype(np.float32))


@pytest.mark.parametrize("Ls", [16, 100])
def test_byte_rows_equal_float_rows_for_float_queries(ssg, built, Ls):
    w, ref, base, g = built
    rng = np.random.default_rng(99)
    q = (w.queries + rng.normal(0.0, 3.3, size=w.queries.shape)).astype(np.float32)
    qc = _cuda(q)
    ids8, d28 = g.search(base, qc, 10, Ls)                       # byte rows
    ids32, d232 = ssg.search_adj(base, g.adj, g.deg, g.nav, qc, 10, Ls)  # float rows
    np.testing.assert_array_equal(_np(ids8), _np(ids32))
    np.testing.assert_array_equal(_np(d28), _np(d232))


def test_other_base_takes_float_rows(ssg, built):
    # a different (but equal-valued) device array is searched through its float rows
    w, ref, base, g = built
    other = base.clone()
    ids, d2 = g.search(other, _cuda(w.queries), 10, 40)
    oid, od2, _, _ = oracle.search(w.base, ref["adj"], ref["deg"], ref["nav"], w.queries, 10, 40)
    np.testing.assert_array_equal(_np(ids), oid)
