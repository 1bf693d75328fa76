"""Appended sub-domain points (Sec. 3.1.1) on the GPU against the oracle (needs a GB300 and the library): the
exact points of a stationary body join Omega_0 with weight one and are interpolated with E itself."""

import numpy as np
import pytest

from oracle import ib as oib
from paper_2103_06415_gb300 import workloads as wl

from runners import check_rel, gpu_context, oracle_history, oracle_sim, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


def _stationary_plate(n=9, x0=1.4, y0=0.2, angle=0.3, h=1.0 / 16):
    q = np.arange(n) * h
    return np.stack([x0 + q * np.cos(angle), y0 + q * np.sin(angle)], axis=1)


def _mixed():
    """small_plate's torsional plate in the box and a stationary plate (prescribed surface velocity) appended
    outside it."""
    w = wl.small_plate()
    w["bodies"].append(dict(kind="rigid", pts=_stationary_plate(), ur=np.tile([0.3, -0.1], (9, 1)), appended=True))
    return w


def test_operator_with_appended_points_matches_oracle_columns(lib):
    w = _mixed()
    sim = oracle_sim(w)
    ctx = gpu_context(w)
    sd = sim.sd
    n2 = 2 * sd.n_sd
    assert ctx.stats()["n_sd"] == sd.n_sd
    cols = [sd.n_box, sd.n_box + 4, sd.n_sd + sd.n_box + 8, 17, sd.n_sd + 40]   # appended and box columns
    for c in cols:
        ref = oib.b0_column(sd, c, w["re"], w["dt"])
        got = ctx.operator_entries(np.arange(n2), np.full(n2, c))
        assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref)), c
    ctx.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_mixed_run_matches_oracle(lib, use_graph):
    w = _mixed()
    n = 10
    sim = oracle_sim(w, tol=1e-12)
    ctx = gpu_context(w, tol=1e-12, use_graph=use_graph)
    for _ in range(n):
        sim.step()
    ctx.advance(n)
    assert np.array_equal(ctx.history(0)[:, 5], oracle_history(sim, 0)[:, 5])
    for body in (0, 1):
        h, r = ctx.history(body), oracle_history(sim, body)
        for k in range(5):
            if np.max(np.abs(r[:, k])) > 0:
                check_rel("test_gpu_appended.py:63", h[:, k], r[:, k], 2e-12)
    check_rel("test_gpu_appended.py:64", ctx.field(0, 0), sim.w[0], 1e-12)
    idx, wts = ctx.interp(sim.nb)
    ridx, rw = sim.last_p
    assert np.array_equal(idx[9:, 0], ridx[9:, 0]) and np.all(wts[9:, 0] == 1.0) and np.all(wts[9:, 1:] == 0.0)
    ctx.close()


def test_only_appended_points_equal_the_true_e_comparator(lib):
    """With every body point appended the sub-domain method is the true-E method (oracle pin); on the GPU the
    two paths are different code (dense B0 columns vs conjugate gradients) and agree to the Krylov tolerance."""
    w = wl.small_plate()
    # inside the box: the true-E comparator bounds its body points by Omega_0
    w["bodies"] = [dict(kind="rigid", pts=_stationary_plate(x0=-0.2, y0=-0.3), appended=True)]
    a = gpu_context(w)
    b = gpu_context(w, coupling=1, krylov_tol=1e-14)
    a.advance(8)
    b.advance(8)
    for k in (0, 1):
        check_rel("test_gpu_appended.py:82", a.history(0)[:, k], b.history(0)[:, k], 1e-13)
    check_rel("test_gpu_appended.py:83", a.field(0, 0), b.field(0, 0), 1e-13)


def test_appended_fp32_close_to_fp64(lib):
    w = _mixed()
    out = []
    for prec in (0, 1):
        ctx = gpu_context(w, precision=prec)
        ctx.advance(10)
        out.append((ctx.history(0), ctx.history(1)))
        ctx.close()
    for body in (0, 1):
        for k in (0, 1):
            check_rel("test_gpu_appended.py:96", out[1][body][:, k], out[0][body][:, k], 3e-6)


def test_appended_limits(lib, tmp_path):
    w = _mixed()
    with pytest.raises(lib.FsiError):                    # no sparse B0' with appended points
        gpu_context(w, drop_tol=0.007)
    ctx = gpu_context(w)
    with pytest.raises(lib.FsiError):                    # operator files do not record appended points
        ctx.save_operator(tmp_path / "b0.bin")
    w_out = _mixed()
    w_out["bodies"][1]["pts"] = _stationary_plate(x0=2.9)  # within 2 cells of the right boundary (x = 3)
    with pytest.raises(lib.FsiError):
        gpu_context(w_out)
