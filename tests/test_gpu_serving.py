"""Serving runtime on the GPU: continuous batching of independent runs (include/ibfsi_server.h)."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context

pytestmark = pytest.mark.gpu


def _drain(srv, limit=100000):
    res = []
    for _ in range(limit):
        n = srv.step()
        res += srv.poll()
        if n == 0 and srv.stats()["queued"] == 0:
            break
    return res + srv.poll()


def test_served_run_is_the_same_alone_and_in_the_mix():
    import paper_2103_06415_gb300 as p
    reqs = wl.serving_requests(5, seed=3, sizes=(128, 256), steps=(20, 40))
    _, w0, b0, n0 = reqs[0]
    alone = p.Server(64 << 30)
    alone.submit(w0, b0, n0, tag=1)
    r_alone = {r["tag"]: r for r in _drain(alone)}
    mix = p.Server(64 << 30)
    for k, (_, w, b, n) in enumerate(reqs):
        mix.submit(w, b, n, tag=k + 1)
    r_mix = {r["tag"]: r for r in _drain(mix)}
    assert len(r_mix) == 5 and all(r["status"] == 0 for r in r_mix.values())
    a, m = r_alone[1], r_mix[1]
    for k in ("fx", "fy", "moment", "theta", "phi"):
        assert a[k] == m[k], k                       # bitwise: runs share no device state
    assert a["steps"] == m["steps"] == n0


def test_served_run_equals_a_context_run():
    import paper_2103_06415_gb300 as p
    _, w, b, _ = wl.serving_requests(1, seed=4, sizes=(128,))[0]
    n = 15
    srv = p.Server(16 << 30)
    srv.submit(w, b, n, precision=p.FSI_PREC_FP32)
    res = _drain(srv)[0]
    w = dict(w, bodies=[b])
    ctx = gpu_context(w, precision=p.FSI_PREC_FP32)
    ctx.advance(n)
    fx, fy, mom = ctx.forces(0)
    th, ph = ctx.deflection(0)
    assert (res["fx"], res["fy"], res["moment"], res["theta"], res["phi"]) == (fx, fy, mom, th, ph)
    assert res["p99_step_ms"] >= res["p50_step_ms"] > 0


def test_admission_respects_the_hbm_budget():
    import paper_2103_06415_gb300 as p
    reqs = wl.serving_requests(4, seed=5, sizes=(128,), steps=(10, 12))
    one = 1.2e9                                  # one 128^2 request (~0.9 GB of B0) fits, two do not
    srv = p.Server(int(one))
    for _, w, b, n in reqs:
        srv.submit(w, b, n)
    max_active = 0
    res = []
    while True:
        n_active = srv.step()
        max_active = max(max_active, n_active, srv.stats()["active"])
        res += srv.poll()
        if n_active == 0 and srv.stats()["queued"] == 0:
            break
    assert max_active <= 1
    assert len(res) == 4 and all(r["status"] == 0 for r in res)
    waits = sorted(r["wait_ms"] for r in res)
    assert waits[-1] > waits[0]
