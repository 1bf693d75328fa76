"""The mixed mode (FSI_PREC_MIXED: double level fields, float transforms, the finest level advanced in
increment form) against the FP64 oracle and the FP64 path (needs a GB300 and the library)."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import check_rel, gpu_context, oracle_history, oracle_sim, rel_err

pytestmark = pytest.mark.gpu

MIXED = 2


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


@pytest.mark.parametrize("workload,steps,bound", [("small_plate", 12, 5e-6), ("small_flag", 12, 5e-6),
                                                  ("plate_128", 100, 1e-6)])
def test_mixed_run_matches_oracle(lib, workload, steps, bound):
    """Force and deflection histories of the mixed mode against the FP64 oracle (relative to each history's
    largest magnitude), with the same FSI iteration counts to within one."""
    w = getattr(wl, workload)()
    sim, ctx = oracle_sim(w), gpu_context(w, precision=MIXED)
    for _ in range(steps):
        sim.step()
    ctx.advance(steps)
    hist, ref = ctx.history(0), oracle_history(sim)
    assert np.max(np.abs(hist[:, 5] - ref[:, 5])) <= 1
    for k in (0, 1, 3, 4):
        if np.max(np.abs(ref[:, k])) > 0:
            check_rel("mixed %s hist%d" % (workload, k), hist[:, k], ref[:, k], bound)
    ctx.close()


def test_mixed_multilevel_fields_match_fp64(lib):
    """Three levels with the flag: after 20 steps every level's w and s in the mixed mode agree with the FP64
    path (the finest level's increments and the coarse levels' full float solves)."""
    w = wl.small_flag(nx=64, ny=64, n_levels=3)
    a, b = gpu_context(w, precision=0), gpu_context(w, precision=MIXED)
    a.advance(20)
    b.advance(20)
    for g in range(3):
        check_rel("mixed 3lvl level%d w" % g, b.field(g, 0), a.field(g, 0), 2e-5)
        check_rel("mixed 3lvl level%d s" % g, b.field(g, 1), a.field(g, 1), 2e-5)
    a.close()
    b.close()


def test_mixed_graph_eager_and_resume_are_bitwise(lib, tmp_path):
    """The captured step graph and eager steps give the same bits; n steps + save + load + n steps equal
    2n steps (the increment form restarts from the double fields exactly)."""
    w = wl.small_flag()
    g, e = gpu_context(w, precision=MIXED), gpu_context(w, precision=MIXED, use_graph=False)
    g.advance(10)
    e.advance(10)
    assert np.array_equal(g.history(0), e.history(0))
    assert np.array_equal(g.field(0, 1), e.field(0, 1))
    path = str(tmp_path / "mixed.state")
    r = gpu_context(w, precision=MIXED)
    r.advance(5)
    r.save_state(path)
    r2 = gpu_context(w, precision=MIXED)
    r2.load_state(path)
    r2.advance(5)
    assert np.array_equal(r2.history(0)[-1], g.history(0)[4 + 5])
    assert np.array_equal(r2.field(0, 0), g.field(0, 0))
    for c in (g, e, r, r2):
        c.close()


def test_mixed_fields_set_mid_run_restart_the_full_form(lib):
    """Fields overwritten between steps break -lap_h s = w; the next step takes the full form, so the run
    continues to follow the FP64 path from the same overwritten state."""
    w = wl.small_plate()
    a, b = gpu_context(w, precision=0), gpu_context(w, precision=MIXED)
    a.advance(4)
    b.advance(4)
    f = a.field(0, 0)
    f[10:20, 10:20] += 0.5
    s0 = a.field(0, 1)
    for c in (a, b):
        c.set_field(0, 0, f)
        c.set_field(0, 1, s0)
        c.advance(6)
    check_rel("mixed after set_field hist0", b.history(0)[:, 0], a.history(0)[:, 0], 1e-5)
    check_rel("mixed after set_field s", b.field(0, 1), a.field(0, 1), 1e-5)
    a.close()
    b.close()


def test_mixed_rejects_tensor_core_transforms_and_true_e(lib):
    w = wl.small_plate()
    with pytest.raises(lib.FsiError):
        lib.Context(128, 128, 1, -1.0, -2.0, 1.0 / 32, 100.0, 0.002, precision=MIXED, dst_method=1)
    c = gpu_context(w, precision=MIXED, coupling=1, precompute=False)
    with pytest.raises(lib.FsiError):
        c.precompute()
    c.close()
