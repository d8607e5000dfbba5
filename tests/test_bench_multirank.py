"""The benchmark's N > 1 path (replicas, no data-path collective): the job time is the
slowest rank's, and the whole-job build time per million points divides it by the points
all ranks built.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    step_ms = [1000.0, 1200.0] if rank == 0 else [3000.0, 3000.0]   # rank 1 is slower
    value, worst = bench.aggregate(step_ms, 1_000_000, ws)
    m = bench.reduce_max([float(rank), 5.0 - rank], ws)
    q.put((rank, value, worst, m))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, worst, m in out:
        assert worst == pytest.approx(3000.0)
        # 3 s for the slowest rank over 2 x 1M points built -> 1.5 s per million
        assert value == pytest.approx(1.5)
        assert m == [1.0, 5.0]


def test_single_rank_identity():
    import bench
    value, worst = bench.aggregate([500.0, 700.0], 2_000_000, 1)
    assert worst == pytest.approx(600.0)
    assert value == pytest.approx(0.3)
