"""The multi-GPU path of bench.py on CPU: two gloo ranks, each with its own workload
(weak scaling, no collective on the data path), timings reduced by MAX, the
whole-job throughput counted over every rank's points."""
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


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 0.5 + rank  # rank 1 is slower
    m = bench.max_over_ranks(local, world)
    v = bench.job_throughput(1000, world, m)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, m, v))


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == pytest.approx(0.5 + (world - 1))  # the slowest rank
        assert v == pytest.approx(world * 1000 / (0.5 + world - 1))


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(0.25, 1) == 0.25
    assert bench.job_throughput(10, 1, 0.5) == 20
