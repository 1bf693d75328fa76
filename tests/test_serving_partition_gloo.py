"""Serving across ranks on CPU: two gloo ranks take disjoint, balanced shares of one request stream
(paper_2103_06415_gb300.serving.partition_requests) and rank 0 aggregates their records as the N > 1 serving
bench does (work summed, the slowest rank's time, latencies pooled)."""

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
    from paper_2103_06415_gb300 import serving
    from paper_2103_06415_gb300 import workloads as wl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    reqs = wl.serving_requests(40, steps=(200, 400))
    mine = serving.partition_requests(reqs, world, rank)
    plans = [None] * world
    dist.all_gather_object(plans, mine)
    cost = sum(serving.request_cost(reqs[k][1], reqs[k][3]) for k in mine)
    local = {"cell_steps": cost, "wall": 1.0 + rank, "finished": len(mine), "errors": 0, "max_active": 3 + rank,
             "ticks": 10, "p50": [0.5 + rank], "p99": [1.0 + rank], "wait": [2.0]}
    parts = bench.gather_serving(local, world)
    agg = bench.aggregate_serving(parts)
    q.put((rank, plans, mine, agg))
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_one_request_stream():
    import torch.multiprocessing as mp

    from paper_2103_06415_gb300 import serving
    from paper_2103_06415_gb300 import workloads as wl
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
    reqs = wl.serving_requests(40, steps=(200, 400))
    plans0, plans1 = out[0][1], out[1][1]
    assert plans0 == plans1                                    # every rank derives the same plan
    a, b = set(plans0[0]), set(plans0[1])
    assert not a & b and a | b == set(range(len(reqs)))        # disjoint and complete
    for r in (0, 1):
        assert out[r][2] == sorted(out[r][2])                  # a rank serves its share in arrival order
    loads = serving.rank_loads(reqs, 2)
    costs = [serving.request_cost(w, n) for _, w, _, n in reqs]
    assert max(loads) <= sum(costs) / 2 + max(costs)           # greedy list-scheduling bound
    for rank, _, _, agg in out:
        assert agg["cell_steps"] == pytest.approx(sum(costs))
        assert agg["wall"] == 2.0 and agg["value"] == pytest.approx(sum(costs) / 2.0)
        assert agg["finished"] == len(reqs) and agg["max_active"] == 4
        assert sorted(agg["p50"]) == [0.5, 1.5]


def test_partition_of_one_rank_is_the_whole_stream_and_bad_ranks_are_rejected():
    from paper_2103_06415_gb300 import serving
    from paper_2103_06415_gb300 import workloads as wl
    reqs = wl.serving_requests(7)
    assert serving.partition_requests(reqs, 1, 0) == list(range(7))
    with pytest.raises(ValueError):
        serving.partition_requests(reqs, 2, 2)
