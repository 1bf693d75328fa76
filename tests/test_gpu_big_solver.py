"""The distributed small-system solver of the FSI kernel (fsi_solver 2: block-Jacobi float inverse and K in
global memory, owned rows exchanged through global memory) against the oracle and against the shared-memory
solver (needs a GB300 and the library)."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import check_rel, gpu_context, oracle_history, oracle_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


@pytest.mark.parametrize("workload", ["small_plate", "small_flag", "small_mixed_bodies", "tandem_small"])
def test_distributed_solver_matches_oracle(lib, workload):
    """Forced on small systems: the same FSI iterations and histories as the oracle at FSI tolerance 1e-12
    (one block for one body: the block inverse is the inverse of K; several bodies in one box are coupled
    through B0 and the refinement against the full K absorbs it)."""
    w = getattr(wl, workload)()
    n = 8
    sim = oracle_sim(w, tol=1e-12)
    for _ in range(n):
        sim.step()
    ctx = gpu_context(w, tol=1e-12, fsi_solver=2)
    ctx.advance(n)
    nbod = len(w["bodies"])
    assert np.array_equal(ctx.history(0)[:, 5], oracle_history(sim, 0)[:, 5])
    for body in range(nbod):
        hist, ref = ctx.history(body), oracle_history(sim, body)
        for k in (0, 1, 3, 4):
            if np.max(np.abs(ref[:, k])) > 0:
                check_rel("big %s body%d hist%d" % (workload, body, k), hist[:, k], ref[:, k], 1e-11)
    idx, _ = ctx.interp(sim.nb)
    assert np.array_equal(idx, sim.last_p[0])
    ctx.close()


def test_distributed_solver_runs_beyond_shared_memory(lib):
    """nf = 246 (three 41-point bodies in three boxes): the automatic choice is the distributed solver; the run
    matches the oracle, including the inverse's first rebuild from a scaled identity and its refreshes."""
    w = wl.tandem_nf246()
    n = 5
    sim = oracle_sim(w, tol=1e-12)
    for _ in range(n):
        sim.step()
    ctx = gpu_context(w, tol=1e-12)
    ctx.advance(n)
    st = ctx.stats()
    assert st["nf"] == 246 and st["inverse_rebuilds"] >= 1
    assert np.array_equal(ctx.history(0)[:, 5], oracle_history(sim, 0)[:, 5])
    for body in range(3):
        hist, ref = ctx.history(body), oracle_history(sim, body)
        for k in (0, 1, 3, 4):
            check_rel("big nf246 body%d hist%d" % (body, k), hist[:, k], ref[:, k], 1e-11)
    check_rel("big nf246 w", ctx.field(0, 0), sim.w[0], 1e-11)
    ctx.close()


@pytest.mark.parametrize("precision,bound", [(0, 1e-10), (2, 1e-6)])
def test_distributed_solver_agrees_with_shared_memory_solver(lib, precision, bound):
    """The flag of the 512 x 256 x 3 workload (nf = 202) with both solvers over 20 steps at an FSI tolerance of
    1e-12: FP64, and the mixed mode."""
    w = wl.flag_512x256_3lvl()
    out = []
    for solver in (1, 2):
        ctx = gpu_context(w, precision=precision, fsi_solver=solver, tol=1e-12)
        ctx.advance(20)
        out.append(ctx.history(0))
        ctx.close()
    assert np.array_equal(out[0][:, 5], out[1][:, 5])
    for k in (0, 1, 3):
        check_rel("big vs small config2 prec%d hist%d" % (precision, k), out[1][:, k], out[0][:, k], bound)


def _plate_201():
    """A 201-point torsional plate at ds = h = 1/200 (chord 1, 20 degrees: the first plate of the 5-level
    1536 x 768 tandem workload) on one level of 384 x 256 cells, Omega_0 [-0.1, 1.1] x [-0.1, 0.5], B0'
    filtered at eps = 0.007: nf = 402, beyond the shared-memory solver."""
    h = 1.0 / 200
    return dict(name="plate_201_sparse", nx=384, ny=256, n_levels=1, x0=-0.3, y0=-0.64, h=h, re=1000.0, dt=2e-4,
                uinf=(1.0, 0.0), steps=2, sd_box=(-0.1, 1.1, -0.1, 0.5), ds=h, drop_tol=0.007,
                bodies=[dict(kind="torsional", hinge=(0.0, 0.0), theta0=0.0, n_pts=201, inertia=1.0, damping=0.0,
                             stiffness=0.2, theta=np.deg2rad(20.0))])


def test_long_plate_with_filtered_operator_matches_oracle_slip_included(lib):
    """The distributed solver with the filtered B0' on a long plate, against the oracle: histories, and the
    velocity the corrector leaves at the body points.  With the filter the small system is solved with
    K' = (ds/h^2) P B0' P^T while the fluid takes the whole operator, so the body points keep a slip of
    (K - K') f after the corrector (a third of the free stream at the impulsive start of this plate, which
    lies along 201 points at ds = h); both implementations must leave the same one."""
    from oracle import grid as og
    w = _plate_201()
    n = 2
    sim = oracle_sim(w, tol=1e-12, drop_tol=w["drop_tol"])
    slips = []
    for _ in range(n):
        sim.step()
    lev, sd = sim.levels[0], sim.sd
    ctx = gpu_context(w, precision=0, tol=1e-12, fsi_solver=2)
    ctx.advance(n)
    assert np.array_equal(ctx.history(0)[:, 5], oracle_history(sim, 0)[:, 5])
    hist, ref = ctx.history(0), oracle_history(sim, 0)
    for k in (0, 1, 2, 3, 4):
        check_rel("big plate_201 hist%d" % k, hist[:, k], ref[:, k], 1e-10)
    for s_field, p in ((ctx.field(0, 1), ctx.interp(sim.nb)), (sim.s[0], sim.last_p)):
        u, v = og.faces_from_s(s_field, lev)
        e0q = sd.e0(u + w["uinf"][0], v + w["uinf"][1])
        idx, wts = p
        slips.append(np.concatenate([(wts * e0q[idx]).sum(1), (wts * e0q[idx + sd.n_sd]).sum(1)]))
    check_rel("big plate_201 velocity at the body points", slips[0], slips[1], 1e-11)
    ctx.close()
