"""Host-side plan of a request stream across GPUs: independent FSI runs (the serving workload) share nothing,
so N ranks serve disjoint parts of one stream with no collective on the data path.  Every rank computes the
same plan from the same request list; the ranks' results are only aggregated at the end."""


def request_cost(w, n_steps):
    """Work of one run in cell-steps: levels x nx x ny per step, times its steps (the throughput unit)."""
    return float(w["n_levels"]) * w["nx"] * w["ny"] * n_steps


def partition_requests(reqs, world, rank):
    """Indices of the requests rank `rank` of `world` serves, in arrival order.  reqs: [(arrival_s, grid dict,
    body dict, n_steps)].  Longest-processing-time-first: requests by decreasing cost (ties by index) each to
    the least-loaded rank (ties to the lowest rank), which bounds every rank's load by 4/3 of the optimum
    makespan; deterministic, so every rank derives the same plan."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside world of %d" % (rank, world))
    costs = [request_cost(r[1], r[3]) for r in reqs]
    order = sorted(range(len(reqs)), key=lambda k: (-costs[k], k))
    load = [0.0] * world
    owner = [0] * len(reqs)
    for k in order:
        q = min(range(world), key=lambda i: (load[i], i))
        owner[k] = q
        load[q] += costs[k]
    return [k for k in range(len(reqs)) if owner[k] == rank]


def rank_loads(reqs, world):
    """Cost assigned to each rank by partition_requests."""
    return [sum(request_cost(reqs[k][1], reqs[k][3]) for k in partition_requests(reqs, world, r))
            for r in range(world)]
