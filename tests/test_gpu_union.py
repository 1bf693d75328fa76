"""Omega_0 as a union of boxes (reading R16) and grids of 3 * 2^k cells on the GPU against the oracle (needs a
GB300 and the library)."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import check_rel, gpu_context, oracle_history, oracle_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


def test_union_b0_matches_oracle_columns(lib):
    """Dense B0 of the three-box union (cross-box blocks included) against the oracle's column solves."""
    from oracle import ib as oib
    w = wl.tandem_small()
    ctx, sim = gpu_context(w), oracle_sim(w)
    sd = sim.sd
    assert ctx.stats()["n_sd"] == sd.n_sd
    n2 = 2 * sd.n_sd
    rng = np.random.default_rng(5)
    cols = list(rng.choice(n2, size=10, replace=False)) + [sd.box_off[1], sd.n_sd + sd.box_off[2] + 3]
    for c in cols:
        ref = oib.b0_column(sd, int(c), w["re"], w["dt"])
        got = ctx.operator_entries(np.arange(n2), np.full(n2, c))
        check_rel("union b0 column", got, ref, 1e-12)
    ctx.close()


@pytest.mark.parametrize("drop_tol", [0.0, 0.007])
def test_tandem_run_matches_oracle(lib, drop_tol):
    """Two torsional plates and a flag in three boxes on a 96 x 48 grid (radix-3 transforms) with two levels,
    dense B0 and the filtered B0' of Eq. filtereq: histories of every body, FSI iteration counts and the P map
    against the oracle at an FSI tolerance of 1e-12."""
    w = wl.tandem_small()
    n = 8
    sim = oracle_sim(w, tol=1e-12, drop_tol=drop_tol)
    for _ in range(n):
        sim.step()
    ctx = gpu_context(w, tol=1e-12, drop_tol=drop_tol)
    ctx.advance(n)
    assert np.array_equal(ctx.history(0)[:, 5], oracle_history(sim, 0)[:, 5])
    for body in range(3):
        hist, ref = ctx.history(body), oracle_history(sim, body)
        for k in (0, 1, 3, 4):
            check_rel("tandem eps=%g body%d hist%d" % (drop_tol, body, k), hist[:, k], ref[:, k], 1e-11)
    idx, wts = ctx.interp(sim.nb)
    ridx, rw = sim.last_p
    assert np.array_equal(idx, ridx)
    assert np.max(np.abs(wts - rw)) < 1e-13
    for g in range(2):
        check_rel("tandem eps=%g level%d w" % (drop_tol, g), ctx.field(g, 0), sim.w[g], 1e-11)
    ctx.close()


def test_union_of_adjacent_boxes_equals_merged_box(lib):
    """Two boxes that tile a larger one, a plate in one and a flag in the other (coupled through the cross-box
    blocks of B0): the same run as with the larger box (points renumbered, K summed in another order: equal
    to rounding)."""
    w = wl.tandem_small()
    flag = dict(w["bodies"][2], clamp=(0.9, 0.0))
    w["bodies"] = [w["bodies"][0], flag]
    w["sd_box"] = [(-0.2, 0.7, -0.6, 0.6), (0.75, 1.6, -0.6, 0.6)]   # vertex columns 13..27 and 28..41
    a = gpu_context(w, tol=1e-12)
    b = gpu_context(dict(w, sd_box=(-0.2, 1.6, -0.6, 0.6)), tol=1e-12)
    assert a.stats()["n_sd"] == b.stats()["n_sd"]
    a.advance(6)
    b.advance(6)
    for body in (0, 1):
        for k in (0, 1, 3):
            check_rel("adjacent boxes body%d hist%d" % (body, k), a.history(body)[:, k], b.history(body)[:, k],
                      1e-12)
    a.close()
    b.close()


def test_union_limits(lib, tmp_path):
    w = wl.tandem_small()
    c = gpu_context(w, precompute=False)
    with pytest.raises(lib.FsiError):                       # boxes sharing vertices
        c.set_subdomain_boxes([(-0.2, 0.7, -0.6, 0.6), (0.6, 1.5, -0.6, 0.6)])
    c.close()
    c = gpu_context(w, b0_method=1, precompute=False)      # column solves: one box only
    with pytest.raises(lib.FsiError):
        c.precompute()
    c.close()
    c = gpu_context(w)
    with pytest.raises(lib.FsiError):                       # operator files record one box
        c.save_operator(str(tmp_path / "op.bin"))
    c.close()
