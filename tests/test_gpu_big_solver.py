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
