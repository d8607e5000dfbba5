"""The small float configuration at its full size: N = 10,000 x 32 from 16 Gaussians
(centres N(0, 4I), unit spread), exact kNN graph K = 20, L = 100, R = 32, alpha = 60, 3
navigating nodes, 1,000 queries.  The whole graph equals the oracle's, and recall@10 at
L_search 10, 20, 40 and 80 is within 0.002 of the oracle's search of the oracle's graph."""
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


@pytest.fixture(scope="module")
def cfg():
    w = synth.small()  # 10,000 x 32, 1,000 queries
    nav = synth.nav_ids(w.n, w.n_nav, 101)
    ref = oracle.build_graph(w.base, w.K, w.L, w.R, w.alpha, nav)
    truth, _ = oracle.knn_queries(w.base, w.queries, 10)
    return w, nav, ref, truth


def test_graph_equals_oracle(ssg, cfg):
    w, nav, ref, truth = cfg
    g = ssg.build(torch.from_numpy(w.base).cuda(), w.K, w.L, w.R, w.alpha, nav=nav)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(g.deg.cpu().numpy(), ref["deg"])
    np.testing.assert_array_equal(g.adj.cpu().numpy(), ref["adj"])


@pytest.mark.parametrize("Ls", [10, 20, 40, 80])
def test_recall_within_tolerance(ssg, cfg, Ls):
    w, nav, ref, truth = cfg
    b = torch.from_numpy(w.base).cuda()
    ids, _ = ssg.search_adj(b, torch.from_numpy(ref["adj"]).cuda(),
                            torch.from_numpy(ref["deg"]).cuda(), torch.from_numpy(nav).cuda(),
                            torch.from_numpy(w.queries).cuda(), 10, Ls)
    torch.cuda.synchronize()
    oids = oracle.search(w.base, ref["adj"], ref["deg"], nav, w.queries, 10, Ls)[0]
    r_gpu = oracle.recall_at(ids.cpu().numpy(), truth, 10)
    r_ora = oracle.recall_at(oids, truth, 10)
    assert abs(r_gpu - r_ora) <= 0.002
