"""Tensor-core sine-matrix GEMM passes (compensated 3xTF32 on tcgen05) against the FP64 oracle, against the
FP32 FFT passes, and inside multi-level runs with boundary-ring terms; the per-pass autotuner."""

import numpy as np
import pytest

from oracle import grid as og
from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context, oracle_history, oracle_sim, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nx,ny", [(128, 128), (256, 128), (128, 512), (512, 256), (1024, 512)])
def test_gemm_level_solve_matches_oracle(nx, ny):
    import paper_2103_06415_gb300 as p
    h, re, dt = 1.0 / nx, 150.0, 0.003
    rhs = wl.random_rhs(ny - 1, nx - 1, seed=nx * 7 + ny)
    w, s = p.level_solve(rhs, h, re, dt, precision=p.FSI_PREC_FP32, dst_method=1)
    wf, sf = p.level_solve(rhs, h, re, dt, precision=p.FSI_PREC_FP32, dst_method=0)
    lev = og.Level(nx, ny, h, 0.0, 0.0)
    zero = np.zeros(lev.shape)
    w_ref = og.solve_aw(rhs, zero, lev, re, dt)
    s_ref = og.solve_lap(w_ref, zero, lev)
    ew, es = rel_err(w, w_ref), rel_err(s, s_ref)
    print("gemm %dx%d: w %.2e s %.2e | fft w %.2e s %.2e" % (nx, ny, ew, es, rel_err(wf, w_ref), rel_err(sf, s_ref)))
    assert ew < 2e-5 and es < 2e-5


@pytest.mark.parametrize("dst_method", [1, 2])
def test_gemm_passes_in_multilevel_steps(dst_method):
    """Three levels of 128 x 128 with random fields: the ring terms of the nested levels enter the
    spectral step of the GEMM y pass; FP32 fields after 3 steps against the FP64 oracle."""
    import paper_2103_06415_gb300 as p
    nx = ny = 128
    levels = 3
    w_desc = dict(nx=nx, ny=ny, n_levels=levels, x0=-1.0, y0=-1.0, h=1.0 / 64, re=200.0, dt=0.004,
                  uinf=(1.0, 0.25), bodies=[], ds=1.0 / 64, sd_box=None)
    sim = oracle_sim(w_desc)
    ctx = p.Context(nx, ny, levels, -1.0, -1.0, 1.0 / 64, 200.0, 0.004, (1.0, 0.25), precision=p.FSI_PREC_FP32,
                    dst_method=dst_method)
    st = ctx.stats()
    print("dst_gemm", st["dst_gemm"], "timings us", st["dst_us"])
    if dst_method == 1:
        assert st["dst_gemm"] == [1, 1, 1]
    for g in range(levels):
        w0 = wl.random_field((ny + 1, nx + 1), seed=100 + g)
        s0 = wl.random_field((ny + 1, nx + 1), seed=200 + g) * 0.1
        if g == levels - 1:
            w0[0, :] = w0[-1, :] = w0[:, 0] = w0[:, -1] = 0.0
            s0[0, :] = s0[-1, :] = s0[:, 0] = s0[:, -1] = 0.0
        sim.w[g][:] = w0
        sim.s[g][:] = s0
        ctx.set_field(g, 0, w0)
        ctx.set_field(g, 1, s0)
    for _ in range(3):
        sim.step()
    ctx.advance(3)
    for g in range(levels):
        assert rel_err(ctx.field(g, 0), sim.w[g]) < 2e-5, g
        assert rel_err(ctx.field(g, 1), sim.s[g]) < 2e-5, g


def test_gemm_passes_in_coupled_run():
    """plate_128 with every sine transform on the tensor cores: force and angle histories against
    the FP64 oracle, at the bound of the FP32 FFT path."""
    import paper_2103_06415_gb300 as p
    w = wl.plate_128()
    sim = oracle_sim(w)
    ctx = p.Context(w["nx"], w["ny"], w["n_levels"], w["x0"], w["y0"], w["h"], w["re"], w["dt"], w["uinf"],
                    precision=p.FSI_PREC_FP32, dst_method=1)
    b = w["bodies"][0]
    ctx.add_torsional(b["hinge"], b["theta0"], b["n_pts"], w["ds"], b["inertia"], b["damping"], b["stiffness"],
                      b["theta"])
    ctx.set_subdomain(*w["sd_box"])
    ctx.precompute()
    n = 40
    for _ in range(n):
        sim.step()
    ctx.advance(n)
    hist, ref = ctx.history(0), oracle_history(sim)
    errs = [np.linalg.norm(hist[:, k] - ref[:, k]) / np.linalg.norm(ref[:, k]) for k in range(4)]
    print("gemm-dst relative L2 errors fx fy moment theta:", errs)
    assert max(errs) < 1e-3


def test_gemm_unsupported_cases_are_reported():
    import paper_2103_06415_gb300 as p
    rhs = wl.random_rhs(63, 63, seed=1)
    with pytest.raises(p.FsiError):                 # 64 x 64 is below the tensor-core tile
        p.level_solve(rhs, 1 / 64, 100.0, 0.01, precision=p.FSI_PREC_FP32, dst_method=1)
    rhs = wl.random_rhs(1023, 1023, seed=1)
    with pytest.raises(p.FsiError):                 # y transforms longer than 512 are FFT only
        p.level_solve(rhs, 1 / 1024, 100.0, 0.01, precision=p.FSI_PREC_FP32, dst_method=1)
    rhs = wl.random_rhs(127, 127, seed=1)
    with pytest.raises(p.FsiError):                 # FP64 has no tensor-core path
        p.level_solve(rhs, 1 / 128, 100.0, 0.01, precision=p.FSI_PREC_FP64, dst_method=1)
    w, _ = p.level_solve(rhs, 1 / 128, 100.0, 0.01, precision=p.FSI_PREC_FP64, dst_method=2)   # falls back
    assert np.all(np.isfinite(w))
