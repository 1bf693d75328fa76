"""Pins for Omega_0 as a union of vertex boxes (reading R16: one box per body, B0 with the cross-box blocks,
so that the bodies stay implicitly coupled).

A union of two boxes that together tile a larger box is that larger box with its points renumbered, so its
B0 (Eq. action) must be the larger box's B0 permuted -- cross-box blocks included -- and its P rows (Eq.
weights) the larger box's rows with the indices mapped; a coupled run with a body in each box must follow
the single-box run to rounding.  Unions of separated boxes keep B0 symmetric positive semi-definite.
"""

import numpy as np
import pytest

from oracle import fsi, grid, ib

LEV = grid.Level(40, 24, 1.0 / 16, -1.0, -0.75)
RE, DT = 100.0, 0.004


def _perm(union, merged):
    """Index of every union point in the merged box's numbering (both components)."""
    pos = {(i, j): k for k, (i, j) in enumerate(zip(merged.pi, merged.pj))}
    p = np.array([pos[(i, j)] for i, j in zip(union.pi, union.pj)])
    return np.concatenate([p, p + merged.n_sd])


def test_union_of_adjacent_boxes_is_the_merged_box_renumbered():
    union = ib.Subdomain(LEV, 0, 0, 0, 0, boxes=[(3, 9, 4, 12), (10, 15, 4, 12)])
    merged = ib.Subdomain(LEV, 3, 15, 4, 12)
    assert union.n_sd == merged.n_sd == 13 * 9
    perm = _perm(union, merged)
    rng = np.random.default_rng(3)
    cols = rng.choice(2 * union.n_sd, size=12, replace=False)
    cols = np.concatenate([cols, [5, union.n_sd + 70]])          # one column per box and component at least
    for c in cols:
        bu = ib.b0_column(union, int(c), RE, DT)
        bm = ib.b0_column(merged, int(perm[c]), RE, DT)
        assert np.max(np.abs(bu - bm[perm])) <= 1e-15 * np.max(np.abs(bm)), c
    # P rows: points inside the cells of either box
    pts = np.array([[LEV.x0 + 4.3 * LEV.h, LEV.y0 + 6.7 * LEV.h], [LEV.x0 + 12.5 * LEV.h, LEV.y0 + 10.1 * LEV.h],
                    [LEV.x0 + 8.9 * LEV.h, LEV.y0 + 11.2 * LEV.h]])
    iu, wu = union.p_rows(pts)
    im, wm = merged.p_rows(pts)
    assert np.array_equal(perm[iu], im)
    assert np.array_equal(wu, wm)


def test_union_needs_the_point_inside_one_box():
    union = ib.Subdomain(LEV, 0, 0, 0, 0, boxes=[(3, 9, 4, 12), (10, 15, 4, 12)])
    with pytest.raises(ValueError):                 # the cell between the boxes belongs to neither
        union.p_rows(np.array([[LEV.x0 + 9.5 * LEV.h, LEV.y0 + 8.0 * LEV.h]]))
    with pytest.raises(ValueError):                 # boxes sharing vertices are rejected
        ib.Subdomain(LEV, 0, 0, 0, 0, boxes=[(3, 9, 4, 12), (9, 15, 4, 12)])


def test_union_b0_symmetric_psd_with_cross_blocks():
    union = ib.Subdomain(LEV, 0, 0, 0, 0, boxes=[(3, 7, 4, 9), (12, 16, 14, 19), (25, 30, 5, 10)])
    b = ib.b0_dense(union, RE, DT)
    assert np.max(np.abs(b - b.T)) < 1e-13 * np.max(np.abs(b))
    assert np.min(np.linalg.eigvalsh(0.5 * (b + b.T))) > -1e-12 * np.max(np.abs(b))
    off = union.box_off
    cross = b[off[0]:off[1], off[1]:off[2]]         # x-components of box 0 against box 1
    assert np.max(np.abs(cross)) > 1e-6 * np.max(np.abs(b))   # the boxes are coupled


def test_run_with_a_body_in_each_box_follows_the_merged_box():
    """A torsional plate in one box and a flag in the other: the union run and the merged-box run agree."""
    from oracle import beam
    h = LEV.h

    def bodies():
        return [fsi.TorsionalBody((LEV.x0 + 5.2 * h, LEV.y0 + 8.1 * h), 0.0, 4, h, 0.05, 0.0, 0.5, 0.2),
                beam.Beam((LEV.x0 + 11.3 * h, LEV.y0 + 8.2 * h), 0.1, 3, h, 0.1, 1e-3, 1e3, tip_angle=0.1)]

    def run(sd_box):
        sim = fsi.Sim(LEV.nx, LEV.ny, h, LEV.x0, LEV.y0, 1, RE, DT, (1.0, 0.0), sd_box, bodies(), h, tol=1e-12)
        for _ in range(4):
            sim.step()
        return sim

    x = lambda i: LEV.x0 + i * h   # noqa: E731
    y = lambda j: LEV.y0 + j * h   # noqa: E731
    u = run([(x(3), x(9), y(4), y(12)), (x(10), x(15), y(4), y(12))])
    m = run((x(3), x(15), y(4), y(12)))
    for ru, rm in zip(u.history, m.history):
        assert ru["iters"] == rm["iters"]
        for bu, bm in zip(ru["bodies"], rm["bodies"]):
            for k in ("fx", "fy", "theta", "phi"):
                assert abs(bu[k] - bm[k]) <= 1e-12 * max(1.0, abs(bm[k])), k
    assert np.max(np.abs(u.w[0] - m.w[0])) <= 1e-12 * np.max(np.abs(m.w[0]))
