"""Offline stage on the GPU: B0 by one DST solve per column (Algorithm 1) in FP64 and FP32, agreement of
the two assembly methods, and the FP64 Cholesky factor of B0 + tau I (config 3 sizes included)."""

import numpy as np
import pytest

from oracle import ib as oib
from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context, oracle_sim

pytestmark = pytest.mark.gpu


def _col_err(ctx, sim, cols):
    n2 = 2 * sim.sd.n_sd
    worst = 0.0
    for c in cols:
        ref = oib.b0_column(sim.sd, int(c), sim.re, sim.dt)
        got = ctx.operator_entries(np.arange(n2), np.full(n2, c))
        worst = max(worst, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
    return worst


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_b0_by_column_solves_matches_oracle(prec, tol):
    for w in (wl.small_plate(), wl.plate_128()):
        ctx, sim = gpu_context(w, precision=prec, b0_method=1), oracle_sim(w)
        cols = np.random.default_rng(5).choice(2 * sim.sd.n_sd, size=12, replace=False)
        assert _col_err(ctx, sim, cols) < tol
        ctx.close()


def test_b0_methods_agree_on_every_entry():
    w = wl.small_plate()
    a, b = gpu_context(w, b0_method=0), gpu_context(w, b0_method=1)
    n2 = 2 * a.stats()["n_sd"]
    r, c = np.meshgrid(np.arange(n2), np.arange(n2), indexing="ij")
    ea = a.operator_entries(r.ravel(), c.ravel())
    eb = b.operator_entries(r.ravel(), c.ravel())
    assert np.max(np.abs(ea - eb)) < 1e-12 * np.max(np.abs(ea))
    B = ea.reshape(n2, n2)
    assert np.max(np.abs(B - B.T)) < 1e-13 * np.max(np.abs(B))


def test_factor_of_shifted_b0_matches_library_cholesky():
    w = wl.small_plate()
    ctx, sim = gpu_context(w), oracle_sim(w)
    n2 = 2 * sim.sd.n_sd
    tau, _ = ctx.factor_operator(tau_rel=1e-6)
    b0 = oib.b0_dense(sim.sd, sim.re, sim.dt)
    ref = np.linalg.cholesky(0.5 * (b0 + b0.T) + tau * np.eye(n2))
    assert abs(tau - 1e-6 * np.max(np.diag(b0))) < 1e-12 * tau
    r, c = np.meshgrid(np.arange(n2), np.arange(n2), indexing="ij")
    L = ctx.factor_entries(r.ravel(), c.ravel()).reshape(n2, n2)
    assert np.all(np.triu(L, 1) == 0)
    assert np.max(np.abs(L - ref)) < 1e-8 * np.max(np.abs(ref))


def test_config3_size_b0_columns_and_factor():
    """1024^2 grid, 8192 unknowns: sampled B0 columns (both methods) against the oracle, then the factor's
    backward error on sampled entries of L L^T - (B0 + tau I)."""
    w = wl.b0_1024()
    sim = oracle_sim(w)
    assert sim.sd.n_sd == 4096
    rng = np.random.default_rng(11)
    cols = rng.choice(8192, size=2, replace=False)
    g = gpu_context(w, b0_method=0)
    assert _col_err(g, sim, cols) < 1e-12
    k = gpu_context(w, b0_method=1)
    assert _col_err(k, sim, cols) < 1e-12
    k.close()
    tau, sec = g.factor_operator(tau_rel=1e-10)
    rows = rng.choice(8192, size=6, replace=False)
    worst = 0.0
    bmax = np.max(np.abs(g.operator_entries(np.arange(8192), np.arange(8192))))
    for i in rows:
        li = g.factor_entries(np.full(8192, i), np.arange(8192))
        for j in rows:
            lj = g.factor_entries(np.full(8192, j), np.arange(8192))
            bij = g.operator_entries([i], [j])[0] + (tau if i == j else 0.0)
            worst = max(worst, abs(li @ lj - bij) / bmax)
    print("config-3 factor: tau %.3e, %.3f s, sampled backward error %.2e" % (tau, sec, worst))
    assert worst < 1e-12
