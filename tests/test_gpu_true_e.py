"""The true-E comparator (Sec. 2.2, Sec. 5.1) on the GPU against the oracle's true-E runs (needs a GB300 and the
library).

The oracle builds the small matrix E C (C^T A C)^-1 C^T E^T column by column and solves it directly; the GPU
solves the same system matrix-free by conjugate gradients with one finest-level (C^T A C)^-1 per iteration.
At a tight Krylov tolerance (relative residual 1e-14) and a tight FSI tolerance (1e-10 on max |dtheta|, both
sides) the two runs take the same FSI iterations and agree to the conditioning of the small system times the
FP64 rounding of the fluid solves.
"""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import check_rel, gpu_context, oracle_history, oracle_sim, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


def _rigid_plate(n_pts=9, angle=np.deg2rad(20.0)):
    """small_plate with its plate held fixed at 20 degrees (RIGID points, stationary)."""
    w = wl.small_plate()
    q = np.arange(n_pts) * w["ds"]
    pts = np.stack([q * np.cos(angle), q * np.sin(angle)], axis=1)
    w["bodies"] = [dict(kind="rigid", pts=pts)]
    return w


def _true_runs(w, n, tol=1e-10, ktol=1e-14, use_graph=True, precision=0):
    sim = oracle_sim(w, coupling="true", tol=tol)
    ctx = gpu_context(w, precision=precision, tol=tol, use_graph=use_graph, coupling=1, krylov_tol=ktol)
    for _ in range(n):
        sim.step()
    ctx.advance(n)
    return sim, ctx


@pytest.mark.parametrize("use_graph", [False, True])
def test_true_e_torsional_plate_matches_oracle(lib, use_graph):
    w = wl.small_plate()
    n = 10
    sim, ctx = _true_runs(w, n, use_graph=use_graph)
    hist, ref = ctx.history(0), oracle_history(sim)
    assert np.array_equal(hist[:, 5], ref[:, 5])            # FSI iterations per step
    for k in range(5):                                       # fx, fy, moment, theta, phi
        check_rel("test_gpu_true_e.py:53", hist[:, k], ref[:, k], 4e-12)
    check_rel("test_gpu_true_e.py:54", ctx.field(0, 0), sim.w[0], 2e-12)
    check_rel("test_gpu_true_e.py:55", ctx.field(0, 1), sim.s[0], 2e-12)
    st = ctx.stats()
    assert st["last_krylov_iters"] > 0 and st["krylov_iters_total"] >= st["last_krylov_iters"]
    assert st["launches_per_step"] >= 5 * st["last_krylov_iters"]
    ctx.close()


def test_true_e_rigid_plate_matches_oracle(lib):
    w = _rigid_plate()
    n = 8
    sim, ctx = _true_runs(w, n)
    hist, ref = ctx.history(0), oracle_history(sim)
    assert np.all(hist[:, 5] == 1) and np.all(ref[:, 5] == 1)
    for k in (0, 1):
        check_rel("test_gpu_true_e.py:69", hist[:, k], ref[:, k], 1e-12)
    check_rel("test_gpu_true_e.py:70", ctx.field(0, 0), sim.w[0], 1e-12)
    ctx.close()


def test_true_e_graph_equals_eager(lib):
    """The device-side loops of the graph replay the eager kernels in the same order: identical results."""
    w = wl.small_plate()
    out = []
    for g in (False, True):
        ctx = gpu_context(w, use_graph=g, coupling=1)
        ctx.advance(12)
        out.append((ctx.history(0), ctx.field(0, 0), ctx.stats()["krylov_iters_total"]))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_true_e_default_tolerances_within_iteration_tolerance(lib):
    """Library defaults (Krylov 1e-10, FSI 1e-7) against the oracle's direct solve at the FSI default."""
    w = wl.small_plate()
    n = 10
    sim = oracle_sim(w, coupling="true")
    ctx = gpu_context(w, coupling=1)
    for _ in range(n):
        sim.step()
    ctx.advance(n)
    hist, ref = ctx.history(0), oracle_history(sim)
    assert np.max(np.abs(hist[:, 5] - ref[:, 5])) <= 1
    for k in (0, 1, 3, 4):
        check_rel("test_gpu_true_e.py:100", hist[:, k], ref[:, k], 1e-6)
    ctx.close()


def test_true_e_fp32_fluid_vs_fp64(lib):
    """FP32 fluid solves in the Krylov operator (default tolerance 1e-5) against the FP64 comparator."""
    w = wl.small_plate()
    n = 10
    out = []
    for prec in (0, 1):
        ctx = gpu_context(w, precision=prec, coupling=1)
        ctx.advance(n)
        out.append(ctx.history(0))
        ctx.close()
    for k in (0, 1, 3, 4):
        check_rel("test_gpu_true_e.py:115", out[1][:, k], out[0][:, k], 1e-4)


def test_true_e_close_to_subdomain_on_plate_128(lib):
    """Sec. 5.1 / Table eldgerror: the sub-domain approximation stays within 2 % of the true E in the
    deflection angle and the lift (relative L2 error, Eq. errortheta) once the impulsive start has passed
    (steps 500-1500 of plate_128, t = 1-3)."""
    w = wl.plate_128()
    n = 1500
    hist = []
    for coupling in (0, 1):
        ctx = gpu_context(w, coupling=coupling)
        ctx.advance(n)
        hist.append(ctx.history(0))
        ctx.close()
    sub, tru = hist
    win = slice(500, n)
    for k, bound in ((3, 0.02), (1, 0.02)):                 # theta, lift
        err = np.linalg.norm(sub[win, k] - tru[win, k]) / np.linalg.norm(tru[win, k])
        assert err < bound, (k, err)
    assert np.all(tru[:, 5] <= 6)


def test_true_e_arguments(lib):
    w = wl.small_plate()
    with pytest.raises(lib.FsiError):
        lib.Context(w["nx"], w["ny"], 1, w["x0"], w["y0"], w["h"], w["re"], w["dt"], coupling=2)
    with pytest.raises(lib.FsiError):                      # no sparse B0' in true-E mode
        gpu_context(w, coupling=1, drop_tol=0.007)
    with pytest.raises(lib.FsiError):                      # deformable bodies: sub-domain coupling only
        gpu_context(wl.small_flag(), coupling=1)
    ctx = gpu_context(w, coupling=1)
    ctx.advance(1)
    with pytest.raises(lib.FsiError):                      # no P in true-E mode
        ctx.interp(9)
    with pytest.raises(lib.FsiError):                      # no B0 in true-E mode
        ctx.operator_entries([0], [0])
    ctx.close()
