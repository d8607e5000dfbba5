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
