"""ssg_connect_noalloc: the connectivity step for callers that cannot allocate device
memory while they run (graph capture, fixed-memory serving loops, hosts with their own
allocator).  Its scratch is a fixed array inside the library, so these checks run it
through the C ABI on two calls in a row and compare each result with ssg_connect, which
takes its scratch from the stream-ordered allocator.  Both calls must agree exactly: the
same kernels decide the same edges.  This file is collected last on purpose."""
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


def _noalloc(ssg, base, adj, deg, nav):
    """One call of the allocation-free entry point on copies of adj/deg."""
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
    assert rc == 0, ssg.lib().ssg_last_error()
    torch.cuda.synchronize()
    return a.cpu().numpy(), dg.cpu().numpy(), rep.value


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
