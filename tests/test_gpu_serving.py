"""Serving with continuous batching (ssg_server_*): requests of mixed size, k and L_search
submitted from several host threads are batched as slots and memory free up, and every
result equals the same search run alone (Alg. 1 per query does not depend on its batch)."""
import threading

import numpy as np
import pytest

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
def graph(ssg):
    w = synth.small(n=4_000, nq=800)
    base = torch.from_numpy(w.base).cuda()
    g = ssg.build(base, w.K, w.L, w.R, w.alpha, nav=synth.nav_ids(w.n, w.n_nav, 17))
    return w, base, g


def test_mix_equals_alone(ssg, graph):
    w, base, g = graph
    rng = np.random.default_rng(5)
    reqs = []
    for _ in range(48):
        nq = int(rng.integers(1, 80))
        k = int(rng.choice([1, 10, 100]))
        ls = int(rng.integers(k, 320))
        rows = rng.choice(w.queries.shape[0], size=nq, replace=False)
        reqs.append((np.ascontiguousarray(w.queries[rows]), k, ls))
    srv = ssg.Server(g, base, n_streams=3, max_batch=256, mem_budget_bytes=96 << 10)
    out = [None] * len(reqs)

    def client(idx):
        tickets = [(i, srv.submit(*reqs[i])) for i in idx]
        for i, t in tickets:
            out[i] = srv.wait(t)

    threads = [threading.Thread(target=client, args=(list(range(c, len(reqs), 4)),))
               for c in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    st = srv.stats()
    srv.close()
    assert st["requests_done"] == len(reqs)
    assert st["batches"] >= 2
    for (q, k, ls), (ids, d2, lat) in zip(reqs, out):
        a_ids, a_d2 = ssg.search_adj(base, g.adj, g.deg, g.nav, q, k, ls)
        np.testing.assert_array_equal(ids, a_ids.cpu().numpy())
        np.testing.assert_array_equal(d2, a_d2.cpu().numpy())
        assert lat >= 0.0


def test_admission_limits(ssg, graph):
    w, base, g = graph
    srv = ssg.Server(g, base, n_streams=2, max_batch=64, mem_budget_bytes=16 << 10)
    with pytest.raises(ssg.SSGError):
        srv.submit(w.queries[:65], 10, 20)        # more than max_batch queries
    with pytest.raises(ssg.SSGError):
        srv.submit(w.queries[:60], 100, 200)      # more device bytes than the whole budget
    with pytest.raises(ssg.SSGError):
        srv.submit(w.queries[:4], 20, 10)         # k > L_search
    t = srv.submit(w.queries[:8], 10, 40)
    ids, _, _ = srv.wait(t)
    a_ids, _ = ssg.search_adj(base, g.adj, g.deg, g.nav, w.queries[:8], 10, 40)
    np.testing.assert_array_equal(ids, a_ids.cpu().numpy())
    srv.close()
