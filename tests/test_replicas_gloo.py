"""The N > 1 bench path on CPU: two gloo ranks aggregate their replica timings (max time, summed work)."""

import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)                 # rank 1 is the slower replica
    local_work = 1.0e6 * (rank + 1)
    dist.barrier()
    total_ms, value = bench.aggregate_replicas(local_ms, local_work, world)
    q.put((rank, total_ms, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_replica_timings():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total_ms, value in out:
        assert total_ms == pytest.approx(200.0)
        assert value == pytest.approx(3.0e6 / 0.2)
