"""The N > 1 bench path: independent replicas, max-over-ranks timing (gloo, CPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 100 * (r + 1) ms for 1e9 edges
    rate, ms = bench.whole_job_rate(1e9, 100.0 * (rank + 1), world)
    bench.barrier(world)
    q.put((rank, rate, ms))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_rate_uses_slowest_rank(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = 100.0 * world
    for rank, rate, ms in res:
        assert ms == slowest
        assert rate == pytest.approx(1e9 * world / (slowest * 1e-3))


def test_single_rank_needs_no_process_group():
    import bench
    rate, ms = bench.whole_job_rate(5e8, 250.0, 1)
    assert ms == 250.0 and rate == pytest.approx(2e9)
