"""Failure detection without a GPU fault (ssg_selftest_wait): the bounded mbarrier wait of
the tensor-core pipelines, run against a barrier that nothing completes, gives up at its
limit or when another warp raises the abort flag, and the kernel returns normally, so the
context stays usable; a barrier that completes is waited on without delay."""
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


def test_completed_barrier_is_not_waited_on(ssg):
    ok, ms = ssg.selftest_wait(2)
    assert ok and ms < 100


def test_abort_flag_ends_the_wait(ssg):
    ok, ms = ssg.selftest_wait(1)
    assert not ok and 15 <= ms < 1500


def test_wait_times_out_and_the_context_survives(ssg):
    ok, ms = ssg.selftest_wait(0)
    assert not ok and 1900 <= ms < 5000
    # the same process and context still compute
    w = synth.small(n=500, d=8, nq=0, seed=91)
    ids, _ = ssg.knn(torch.from_numpy(w.base).cuda(), 5)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ids.cpu().numpy(), oracle.knn_rows(w.base, 5)[0])


def test_invalid_mode_rejected(ssg):
    with pytest.raises(ssg.SSGError):
        ssg.selftest_wait(3)


# ---- invariant checks (ssg_build_opts.debug_checks, ssg_check_graph) -------------------
@pytest.fixture(scope="module")
def ref():
    w = synth.small(n=800, d=16, nq=0, seed=93)
    nav = synth.nav_ids(w.n, 3, 95)
    return w, nav, oracle.build_graph(w.base, 10, 40, 12, 60.0, nav)


def test_debug_checks_pass_on_correct_builds(ssg, ref):
    w, nav, o = ref
    b = torch.from_numpy(w.base).cuda()
    g = ssg.build(b, 10, 40, 12, 60.0, nav=nav, debug_checks=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(g.deg.cpu().numpy(), o["deg"])
    np.testing.assert_array_equal(g.adj.cpu().numpy(), o["adj"])
    iw = synth.sift_like(n=3000, nq=0, n_clusters=30)
    g = ssg.build(torch.from_numpy(iw.base).cuda(), 20, 60, 24, 60.0, n_nav=4, debug_checks=True)
    assert ssg.check_graph(g.adj, g.deg) == (-1, 0)


def test_check_graph_reports_each_planted_error(ssg, ref):
    w, nav, o = ref
    adj, deg = o["adj"].copy(), o["deg"].copy()
    assert ssg.check_graph(adj, deg) == (-1, 0)
    R = adj.shape[1]
    rows = [i for i in range(w.n) if 2 <= deg[i] < R]
    a, b, c, e, f = rows[:5]

    def planted(fn):
        x, y = adj.copy(), deg.copy()
        fn(x, y)
        return ssg.check_graph(x, y)

    assert planted(lambda x, y: y.__setitem__(a, R + 1)) == (a, 1)
    assert planted(lambda x, y: x.__setitem__((b, 0), w.n)) == (b, 2)
    assert planted(lambda x, y: x.__setitem__((c, 0), c)) == (c, 3)
    assert planted(lambda x, y: x.__setitem__((e, 1), x[e, 0])) == (e, 4)
    assert planted(lambda x, y: x.__setitem__((f, y[f]), 0)) == (f, 5)

    def several(x, y):
        x[f, 0] = w.n
        x[c, 0] = c
    assert planted(several) == (min(c, f), 3 if c < f else 2)


# ---- injected allocation failures (ssg_debug_fail_alloc, on the host) ------------------
def test_injected_allocation_failure_returns_enomem(ssg, ref):
    w, nav, o = ref
    b = torch.from_numpy(w.base).cuda()
    for nth in (1, 2, 3, 8):
        ssg.debug_fail_alloc(nth)
        try:
            with pytest.raises(ssg.SSGError) as e:
                ssg.build(b, 10, 40, 12, 60.0, nav=nav)
            assert e.value.status == 2 and "injected" in str(e.value)
        finally:
            ssg.debug_fail_alloc(0)
        # what the failed call held was released; the next build is whole and right
        g = ssg.build(b, 10, 40, 12, 60.0, nav=nav)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(g.deg.cpu().numpy(), o["deg"])
        np.testing.assert_array_equal(g.adj.cpu().numpy(), o["adj"])
        del g
