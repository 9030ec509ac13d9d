"""bench.py's multi-rank aggregation on CPU (gloo, world size 2): whole-job
throughput is the units of all ranks over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r processed 100 * (r + 1) units in (r + 1) seconds
    val, tmax = bench.aggregate(100.0 * (rank + 1), float(rank + 1), world)
    bench._barrier(world)
    q.put((rank, val, tmax))
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, val, tmax in res:
        assert tmax == pytest.approx(2.0)
        assert val == pytest.approx(300.0 / 2.0)


def test_aggregate_single_rank():
    import bench
    assert bench.aggregate(50.0, 2.0, 1) == (25.0, 2.0)
