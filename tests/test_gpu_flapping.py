"""The flapping pair of Sec. 5.1 (driven plate with prescribed heave and pitch, passive plate hinged to it
under the pseudo-forces of Eq. newtonseldg) on the GPU against the FP64 oracle (needs a GB300 and the library)."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import check_rel, gpu_context, oracle_history, oracle_sim, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


def _runs(w, n, tol=1e-7, use_graph=True, **kw):
    sim = oracle_sim(w, tol=tol, coupling="true" if kw.get("coupling") == 1 else "subdomain")
    ctx = gpu_context(w, tol=tol, use_graph=use_graph, **kw)
    for _ in range(n):
        sim.step()
    ctx.advance(n)
    return sim, ctx


def _compare(sim, ctx, bound):
    for body in (0, 1):
        hist, ref = ctx.history(body), oracle_history(sim, body)
        for k in range(5):
            if np.max(np.abs(ref[:, k])) > 0:
                check_rel("test_gpu_flapping.py:34", hist[:, k], ref[:, k], bound)
            else:
                assert np.all(hist[:, k] == 0.0), (body, k)


@pytest.mark.parametrize("use_graph", [False, True])
def test_flapping_pair_matches_oracle_at_tight_tolerance(lib, use_graph):
    w = wl.small_flapping()
    n = 12
    sim, ctx = _runs(w, n, tol=1e-12, use_graph=use_graph)
    assert np.array_equal(ctx.history(1)[:, 5], oracle_history(sim, 1)[:, 5])
    _compare(sim, ctx, 1e-12)
    check_rel("test_gpu_flapping.py:46", ctx.field(0, 0), sim.w[0], 1e-12)
    idx, wts = ctx.interp(sim.nb)
    ridx, rw = sim.last_p
    assert np.array_equal(idx, ridx)
    assert np.max(np.abs(wts - rw)) < 1e-12
    ctx.close()


def test_flapping_pair_default_tolerance(lib):
    w = wl.small_flapping()
    n = 12
    sim, ctx = _runs(w, n)
    assert np.max(np.abs(ctx.history(1)[:, 5] - oracle_history(sim, 1)[:, 5])) <= 1
    _compare(sim, ctx, 1e-7)
    ctx.close()


def test_flapping_pair_kinematics_table_wraps(lib):
    """More steps than the kinematics table holds, in uneven advance calls: same history as one call (small
    amplitude, so that the pair stays inside the small grid's Omega_0 for 2.2 periods)."""
    w = wl.small_flapping(a0=0.4, beta=0.3, dt=0.002)
    out = []
    for chunks in ((1100,), (3, 1020, 77)):
        ctx = gpu_context(w)
        for k in chunks:
            ctx.advance(k)
        out.append(ctx.history(1))
        ctx.close()
    assert np.array_equal(out[0], out[1])


def test_flapping_pair_true_e_matches_oracle(lib):
    w = wl.small_flapping()
    n = 8
    sim, ctx = _runs(w, n, tol=1e-10, coupling=1, krylov_tol=1e-14)
    assert np.array_equal(ctx.history(1)[:, 5], oracle_history(sim, 1)[:, 5])
    _compare(sim, ctx, 1e-12)
    ctx.close()


def test_flapping_arguments(lib):
    w = wl.small_flapping()
    c = lib.Context(w["nx"], w["ny"], 1, w["x0"], w["y0"], w["h"], w["re"], w["dt"], (0.0, 0.0))
    with pytest.raises(lib.FsiError):                    # invalid kinematics
        c.add_driven((0, 0), -0.5, 16, w["ds"], 1.4, 0.7, -1.0, 1.0)
    d = c.add_driven((0, 0), -0.5, 16, w["ds"], 1.4, 0.7, 0.628, 0.628)
    with pytest.raises(lib.FsiError):                    # driver must be a driven body that exists
        c.add_torsional((0, 0), 0.0, 17, w["ds"], 0.3, 0.0, 1.0, 0.0, driver=d + 5, hinge_offset=0.55)
    with pytest.raises(lib.FsiError):                    # theta0 must be 0 on a driver
        c.add_torsional((0, 0), 0.1, 17, w["ds"], 0.3, 0.0, 1.0, 0.0, driver=d, hinge_offset=0.55)
    t = c.add_torsional((0, 0), 0.0, 5, w["ds"], 0.3, 0.0, 1.0, 0.0, driver=None)
    with pytest.raises(lib.FsiError):                    # a torsional body is not a driver
        c.add_torsional((0, 0), 0.0, 17, w["ds"], 0.3, 0.0, 1.0, 0.0, driver=t, hinge_offset=0.55)
    c.close()


@pytest.mark.parametrize("case", [1, 2])
def test_e1_flapping_runs_with_few_fsi_iterations(lib, case):
    """The paper's E1 cases (5 levels of 512^2, sparse B0' at eps = 0.007): at most three FSI iterations per
    step (Sec. 5.1), FP32 fluid within 1e-4 of FP64 on the passive plate's angle."""
    w = wl.e1_flapping(case)
    n = 150
    hist = []
    for prec in (0, 1):
        ctx = gpu_context(w, precision=prec, drop_tol=0.007)
        ctx.advance(n)
        hist.append(ctx.history(1))
        ctx.close()
    h64, h32 = hist
    assert np.max(h64[:, 5]) <= 3
    assert np.all(np.isfinite(h64[:, :5]))
    check_rel("test_gpu_flapping.py:117", h32[:, 3], h64[:, 3], 5e-6)
