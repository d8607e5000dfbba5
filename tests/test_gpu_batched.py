"""Batched builds of independent indices (ssg_build_batched): every graph equals the one
ssg_build gives for the same input, bit for bit, and one of them equals the oracle's."""
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


def _inputs():
    """Float mixtures of several shapes plus one integer index (tensor-core paths)."""
    out = []
    for i, (n, d) in enumerate([(800, 16), (3000, 64), (1500, 96), (2200, 33), (4000, 128)]):
        w = synth.small(n=n, d=d, nq=0, seed=4200 + i)
        out.append(w.base)
    out.append(synth.uniform_points(2600, 64, 4299, integer=True, hi=255))
    return out


def _cpu(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("n_streams", [1, 3, 8])
def test_batched_equals_one_by_one(ssg, n_streams):
    bases = [torch.from_numpy(b).cuda() for b in _inputs()]
    K, L, R, alpha = 20, 40, 16, 60.0
    Ls = [40, 60, 40, 30, 40, 50]
    gs = ssg.build_batched(bases, K, Ls, R, alpha, n_streams=n_streams)
    for b, l, g in zip(bases, Ls, gs):
        ref = ssg.build(b, K, l, R, alpha)
        np.testing.assert_array_equal(_cpu(g.deg), _cpu(ref.deg))
        np.testing.assert_array_equal(_cpu(g.adj), _cpu(ref.adj))
        np.testing.assert_array_equal(_cpu(g.nav), _cpu(ref.nav))


def test_batched_matches_oracle(ssg):
    base = synth.small(n=900, d=24, nq=0, seed=4300).base
    other = synth.small(n=1200, d=40, nq=0, seed=4301).base
    gs = ssg.build_batched([torch.from_numpy(base).cuda(), torch.from_numpy(other).cuda()],
                           12, 30, 10, 60.0, n_streams=2)
    nav = _cpu(gs[0].nav)
    ref = oracle.build_graph(base, 12, 30, 10, 60.0, nav)
    np.testing.assert_array_equal(_cpu(gs[0].deg), ref["deg"])
    np.testing.assert_array_equal(_cpu(gs[0].adj), ref["adj"])


def test_wide_rows_in_the_batch(ssg):
    """A 960-d index (kept vectors in a device slot per warp: the second shape class of the
    persistent prune) next to narrow ones."""
    ws = [synth.gist_like(n=700, nq=0, n_clusters=6).base, synth.small(n=900, d=48, nq=0, seed=4310).base]
    bases = [torch.from_numpy(b).cuda() for b in ws]
    gs = ssg.build_batched(bases, 12, 40, 70, 60.0, n_streams=2)
    for b, g in zip(bases, gs):
        ref = ssg.build(b, 12, 40, 70, 60.0)
        np.testing.assert_array_equal(_cpu(g.deg), _cpu(ref.deg))
        np.testing.assert_array_equal(_cpu(g.adj), _cpu(ref.adj))


def test_autotuned_batch_equals_one_by_one(ssg, tmp_path):
    """The autotuner writes a tune table; a batch built with it equals the one-by-one builds
    (launch parameters change the speed, not the graph)."""
    bases = [torch.from_numpy(b).cuda() for b in _inputs()]
    K, L, R, alpha = 20, 40, 16, 60.0
    path = str(tmp_path / "batch_tune.txt")
    prune_ms, knn_ms = ssg.autotune_batched(bases, K, L, R, alpha, path)
    assert prune_ms > 0.0
    text = open(path).read()
    names = {ln.split("=")[0].strip() for ln in text.splitlines() if ln and not ln.startswith("#")}
    assert names == {"prune_warps", "prune_bucket_width", "knn_stream_rows"}
    gs = ssg.build_batched(bases, K, L, R, alpha, n_streams=4, tune_table=path)
    for b, g in zip(bases, gs):
        ref = ssg.build(b, K, L, R, alpha)
        np.testing.assert_array_equal(_cpu(g.deg), _cpu(ref.deg))
        np.testing.assert_array_equal(_cpu(g.adj), _cpu(ref.adj))
    assert all(g.stats["ms_prune"] > 0.0 for g in gs)
