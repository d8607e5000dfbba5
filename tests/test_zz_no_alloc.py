"""ssg_connect_noalloc: the connectivity step for callers that cannot allocate device
memory while they run (serving loops whose device memory is fixed before requests
arrive, hosts with their own allocator).  Its scratch is a fixed array inside the
library, so these checks run it through the C ABI on two calls in a row and compare each
result with ssg_connect, which takes its scratch from the stream-ordered allocator.  Both
calls must agree exactly: the same kernels decide the same edges.  The checks also show
that the call allocates nothing (an injected allocation failure is left for the next
allocating call), that a bad navigating id leaves the graph untouched, and that the limit
on tied nodes is reported.  This file is collected last on purpose."""
import ctypes

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


def _sparse_graph(n, R, seed):
    rng = np.random.default_rng(seed)
    adj = np.full((n, R), -1, np.int32)
    deg = rng.integers(0, 3, size=n).astype(np.int32)
    for i in range(n):
        adj[i, :deg[i]] = rng.choice(n, size=deg[i], replace=False)
    return adj, deg


def _noalloc_rc(ssg, base, adj, deg, nav):
    """One call of the allocation-free entry point on copies of adj/deg: (status, adj, deg,
    repairs)."""
    b = torch.from_numpy(np.ascontiguousarray(base)).cuda()
    a = torch.from_numpy(adj.copy()).cuda()
    dg = torch.from_numpy(deg.copy()).cuda()
    nv = torch.from_numpy(np.asarray(nav, np.int32)).cuda()
    rep = ctypes.c_int64(-1)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = ssg.lib().ssg_connect_noalloc(ctypes.c_void_p(b.data_ptr()), b.shape[0], b.shape[1],
                                       ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(dg.data_ptr()),
                                       a.shape[1], ctypes.c_void_p(nv.data_ptr()), nv.numel(),
                                       ctypes.byref(rep), st)
    torch.cuda.synchronize()
    return rc, a.cpu().numpy(), dg.cpu().numpy(), rep.value


def _noalloc(ssg, base, adj, deg, nav):
    rc, a, dg, rep = _noalloc_rc(ssg, base, adj, deg, nav)
    assert rc == 0, ssg.lib().ssg_last_error()
    return a, dg, rep


@pytest.mark.parametrize("case", ["components", "nssg"])
def test_noalloc_matches_connect_twice(ssg, case):
    if case == "components":
        n, R = 5000, 6
        base = synth.uniform_points(n, 4, 81)
        adj, deg = _sparse_graph(n, R, 9)
        nav = synth.nav_ids(n, 4, 321)
    else:
        w = synth.small(n=4000, nq=1)
        base = w.base
        nav = synth.nav_ids(w.n, w.n_nav, 11)
        b = torch.from_numpy(base).cuda()
        ids, _ = ssg.knn(b, w.K)
        pid, _, pl = ssg.pool(b, ids, w.L)
        adj0, deg0 = ssg.prune(b, pid, pl, w.R, w.alpha)
        adj1, deg1 = ssg.reverse(b, adj0, deg0, w.alpha)
        adj, deg = adj1.cpu().numpy(), deg1.cpu().numpy()
    ref_adj, ref_deg, ref_rep = ssg.connect(torch.from_numpy(base).cuda(), adj, deg, nav)
    ref_adj, ref_deg = ref_adj.cpu().numpy(), ref_deg.cpu().numpy()
    for _ in range(2):   # the shared scratch keeps the previous call's contents
        a, dg, rep = _noalloc(ssg, base, adj, deg, nav)
        assert rep == ref_rep
        np.testing.assert_array_equal(dg, ref_deg)
        np.testing.assert_array_equal(a, ref_adj)
    if case == "components":
        assert ref_rep > 100


def test_noalloc_rejects_sizes_beyond_its_scratch(ssg):
    P = ctypes.c_void_p(256)   # never dereferenced: the size check fails first
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = ssg.lib()
    assert L.ssg_connect_noalloc(P, (1 << 20) + 1, 4, P, P, 8, P, 1, None, st) == 1
    assert b"n <=" in L.ssg_last_error()
    assert L.ssg_connect_noalloc(P, 1000, 6, P, P, 8, P, 1, None, st) == 1


def test_noalloc_allocates_nothing(ssg):
    """With the next scratch allocation set to fail, the allocation-free call still
    succeeds, and the failure is left for the first allocating call after it."""
    n, R = 3000, 6
    base = synth.uniform_points(n, 4, 82)
    adj, deg = _sparse_graph(n, R, 10)
    nav = synth.nav_ids(n, 3, 322)
    b = torch.from_numpy(base).cuda()
    try:
        ssg.debug_fail_alloc(1)
        a, dg, rep = _noalloc(ssg, base, adj, deg, nav)
        assert rep > 0
        with pytest.raises(ssg.SSGError) as e:
            ssg.connect(b, adj, deg, nav)
        assert e.value.status == 2
    finally:
        ssg.debug_fail_alloc(0)
    ref_adj, ref_deg, ref_rep = ssg.connect(b, adj, deg, nav)
    assert rep == ref_rep
    np.testing.assert_array_equal(a, ref_adj.cpu().numpy())


def test_noalloc_bad_navigating_id_leaves_graph(ssg):
    n, R = 2000, 6
    base = synth.uniform_points(n, 4, 83)
    adj, deg = _sparse_graph(n, R, 11)
    rc, a, dg, rep = _noalloc_rc(ssg, base, adj, deg, [0, 5, n + 7])
    assert rc == 1 and b"out of range" in ssg.lib().ssg_last_error()
    np.testing.assert_array_equal(a, adj)
    np.testing.assert_array_equal(dg, deg)


def test_noalloc_reports_too_many_ties(ssg):
    """20,000 reached nodes at one point and one unreached node next to them: all 20,000
    tie for its nearest reached node, more than the 16,384 the fixed array can list, so the
    allocation-free call reports it while ssg_connect (exhaustive search) links the
    smallest id."""
    n, R = 20_001, 4
    base = np.zeros((n, 4), np.float32)
    base[-1, 0] = 1.0
    adj = np.full((n, R), -1, np.int32)
    deg = np.zeros(n, np.int32)
    adj[:n - 2, 0] = np.arange(1, n - 1)   # a chain 0 -> 1 -> ... -> n - 2
    deg[:n - 2] = 1
    rc, a, dg, rep = _noalloc_rc(ssg, base, adj, deg, [0])
    assert rc == 5 and b"tie" in ssg.lib().ssg_last_error()
    ref_adj, ref_deg, ref_rep = ssg.connect(torch.from_numpy(base).cuda(), adj, deg, [0])
    assert ref_rep == 1
    assert ref_adj.cpu().numpy()[0, 1] == n - 1
