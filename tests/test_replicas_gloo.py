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


def _dying_worker(rank, world, port, q):
    """Rank 1 leaves between steps (after the first barrier, before the second); rank 0 must learn of it
    from its next collective, which ends with an error within the short process-group timeout."""
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    dist.barrier()
    if rank == 1:
        q.put((rank, "left"))
        q.close()
        q.join_thread()                    # flush the message, then leave without any cleanup
        os._exit(0)
    try:
        dist.barrier()
        q.put((rank, "no error"))
    except Exception as e:                 # timeout or connection reset, depending on the transport
        q.put((rank, "error: " + type(e).__name__))


def test_a_rank_that_leaves_is_detected_by_the_next_collective():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert out[1] == "left"
    assert out[0].startswith("error"), out[0]
