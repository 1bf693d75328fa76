"""Offline stage on the GPU: B0 by one DST solve per column (Algorithm 1) in FP64 and FP32, agreement of
the two assembly methods, and the FP64 Cholesky factor of B0 + tau I (the b0_1024 sizes included)."""

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
    print("b0_1024 factor: tau %.3e, %.3f s, sampled backward error %.2e" % (tau, sec, worst))
    assert worst < 1e-12


def _set_boxes_small():
    # three boxes of different sizes and positions on a 64 x 64 grid, h = 1/16, corner (-2, -2)
    return [(-1.5, -1.0, -1.5, -0.75), (-0.25, 0.75, 0.0, 0.5), (0.75, 1.625, -1.75, -1.25)]


def test_b0_set_matches_single_box_builds_and_oracle():
    """Several uneven Omega_0 boxes built in one pass equal, box by box, the single-box build (bitwise for
    the Green's-function method) and the oracle's columns; the column-solve method agrees to 1e-12."""
    import paper_2103_06415_gb300 as p
    from oracle import grid as og
    boxes = _set_boxes_small()
    grid = dict(nx=64, ny=64, x0=-2.0, y0=-2.0, h=1.0 / 16, re=100.0, dt=0.004)
    sg = p.B0Set(grid["nx"], grid["ny"], grid["x0"], grid["y0"], grid["h"], grid["re"], grid["dt"], boxes)
    sc = p.B0Set(grid["nx"], grid["ny"], grid["x0"], grid["y0"], grid["h"], grid["re"], grid["dt"], boxes, method=1)
    sf = p.B0Set(grid["nx"], grid["ny"], grid["x0"], grid["y0"], grid["h"], grid["re"], grid["dt"], boxes, method=1,
                 precision=p.FSI_PREC_FP32)
    lev = og.Level(grid["nx"], grid["ny"], grid["h"], grid["x0"], grid["y0"])
    sizes = set()
    for k, b in enumerate(boxes):
        info = sg.box(k)
        sd = oib.Subdomain.from_box(lev, *b)
        assert (info["i_lo"], info["i_hi"], info["j_lo"], info["j_hi"]) == (sd.i_lo, sd.i_hi, sd.j_lo, sd.j_hi)
        n2 = 2 * info["n_sd"]
        sizes.add(n2)
        r, c = np.meshgrid(np.arange(n2), np.arange(n2), indexing="ij")
        g = sg.entries(k, r.ravel(), c.ravel())
        w = dict(grid, name="one", n_levels=1, uinf=(1.0, 0.0), sd_box=b, bodies=[], ds=grid["h"])
        one = gpu_context(w)
        assert np.array_equal(g, one.operator_entries(r.ravel(), c.ravel()))
        one.close()
        scale = np.max(np.abs(g))
        assert np.max(np.abs(sc.entries(k, r.ravel(), c.ravel()) - g)) < 1e-12 * scale
        assert np.max(np.abs(sf.entries(k, r.ravel(), c.ravel()) - g)) < 2e-5 * scale
        G = g.reshape(n2, n2)
        for col in (0, n2 // 2 + 1, n2 - 1):
            ref = oib.b0_column(sd, col, grid["re"], grid["dt"])
            assert np.max(np.abs(G[:, col] - ref)) < 1e-12 * np.max(np.abs(ref))
    assert len(sizes) == 3
    for s in (sg, sc, sf):
        s.close()


def test_config3_sixteen_uneven_subdomains_in_one_build():
    """Sixteen boxes of 256 ... 4096 points on the 1024^2 grid (h = 1/256, Re 500, dt = h/4), built together by
    both methods: sampled columns of the smallest, a middle and the largest box against the oracle."""
    import paper_2103_06415_gb300 as p
    from oracle import grid as og
    w = wl.b0_1024()
    boxes = wl.b0_1024_uneven_boxes()
    args = (w["nx"], w["ny"], w["x0"], w["y0"], w["h"], w["re"], w["dt"], boxes)
    sg = p.B0Set(*args)
    sf = p.B0Set(*args, method=1, precision=p.FSI_PREC_FP32)
    n_pts = [sg.box(k)["n_sd"] for k in range(16)]
    assert n_pts[0] == 256 and n_pts[-1] == 4096 and len(set(n_pts)) == 16
    lev = og.Level(w["nx"], w["ny"], w["h"], w["x0"], w["y0"])
    rng = np.random.default_rng(13)
    for k in (0, 7, 15):
        sd = oib.Subdomain.from_box(lev, *boxes[k])
        n2 = 2 * sd.n_sd
        for col in rng.choice(n2, size=2, replace=False):
            ref = oib.b0_column(sd, int(col), w["re"], w["dt"])
            got = sg.entries(k, np.arange(n2), np.full(n2, col))
            assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
            f32 = sf.entries(k, np.arange(n2), np.full(n2, col))
            assert np.max(np.abs(f32 - ref)) < 2e-5 * np.max(np.abs(ref))
    print("16 uneven boxes: green %.3f s, columns fp32 %.3f s" % (sg.stats()["seconds"], sf.stats()["seconds"]))
    sg.close()
    sf.close()
