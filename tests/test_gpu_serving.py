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


def _solo_history(w, body, n, precision):
    import paper_2103_06415_gb300 as p
    ctx = gpu_context(dict(w, bodies=[body]), precision=precision)
    ctx.advance(n)
    h = ctx.history(0)
    ctx.close()
    return h


def test_run_admitted_while_others_step_keeps_every_history_bitwise():
    """Two runs start; a third is submitted after they have stepped five times and admitted while they keep
    stepping.  Every run's whole history equals the same run's on a context of its own, bit for bit."""
    import paper_2103_06415_gb300 as p
    reqs = wl.serving_requests(3, seed=7, sizes=(128, 256), steps=(24, 30))
    srv = p.Server(64 << 30)
    ids = {}
    for k, (_, w, b, n) in enumerate(reqs[:2]):
        ids[srv.submit(w, b, n, tag=k, history=True)] = k
    res = []
    for _ in range(5):
        srv.step()
        res += srv.poll()
    st = srv.stats()
    assert st["active"] == 2 and not res
    _, w3, b3, n3 = reqs[2]
    ids[srv.submit(w3, b3, n3, tag=2, history=True)] = 2
    res += _drain(srv)
    assert len(res) == 3 and all(r["status"] == 0 for r in res)
    for r in res:
        _, w, b, n = reqs[r["tag"]]
        want = _solo_history(w, b, n, p.FSI_PREC_FP32)
        assert r["history"].shape == want.shape
        assert np.array_equal(r["history"], want), r["tag"]
    srv.close()


def test_served_flag_equals_a_context_run():
    """A deformable body (the clamped flag of App. A) served, against a context run: the whole history."""
    import paper_2103_06415_gb300 as p
    w = wl.small_flag()
    body = w["bodies"][0]
    n = 12
    srv = p.Server(16 << 30)
    srv.submit(w, body, n, precision=p.FSI_PREC_FP64, history=True)
    res = _drain(srv)[0]
    assert res["status"] == 0 and res["steps"] == n
    want = _solo_history(w, body, n, p.FSI_PREC_FP64)
    assert np.array_equal(res["history"], want)
    srv.close()


def test_resident_runs_step_while_a_newcomer_is_admitted():
    """The operator of a newcomer (a 1024^2 grid) is built on the server's worker thread: meanwhile every tick
    still advances the resident run by one step."""
    import paper_2103_06415_gb300 as p
    small = wl.serving_requests(1, seed=8, sizes=(128,), steps=(4000, 4000))[0]
    big = wl.serving_requests(1, seed=9, sizes=(1024,), steps=(3, 3))[0]
    srv = p.Server(64 << 30)
    srv.submit(small[1], small[2], small[3], tag=0)
    while srv.stats()["active"] < 1:
        srv.step()
    srv.submit(big[1], big[2], big[3], tag=1)
    ticks_while_admitting = 0
    steps0 = srv.stats()["run_steps"]
    for _ in range(20000):
        srv.step()
        st = srv.stats()
        if st["admitting"] == 0:
            break
        ticks_while_admitting += 1
    assert ticks_while_admitting >= 2
    assert srv.stats()["run_steps"] - steps0 >= ticks_while_admitting   # the resident run kept stepping
    srv.close()
