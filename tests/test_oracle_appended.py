"""Pins of the oracle's appended sub-domain points (Sec. 3.1.1: the exact points of stationary bodies join
Omega_0 with weight one and are interpolated with E itself)."""

import numpy as np

from oracle import grid as ogrid
from oracle import ib
from paper_2103_06415_gb300 import workloads as wl

from runners import oracle_history, oracle_sim


def _stationary_plate(n=9, x0=1.4, y0=0.2, angle=0.3, h=1.0 / 16):
    q = np.arange(n) * h
    return np.stack([x0 + q * np.cos(angle), y0 + q * np.sin(angle)], axis=1)


def test_only_appended_bodies_equal_the_true_e_run():
    """With every body point appended, P B0 P^T is E C (C^T A C)^-1 C^T E^T at the points, the right-hand side
    E (C s* + q_inf) and the corrector E^T f: the sub-domain run is the true-E run."""
    w = wl.small_plate()
    w["bodies"] = [dict(kind="rigid", pts=_stationary_plate(), appended=True)]
    a = oracle_sim(w)
    b = oracle_sim(w, coupling="true")
    for _ in range(4):
        a.step()
        b.step()
    ha, hb = oracle_history(a), oracle_history(b)
    for k in (0, 1):
        assert np.max(np.abs(ha[:, k] - hb[:, k])) < 1e-11 * np.max(np.abs(hb[:, k])), k
    assert np.max(np.abs(a.w[0] - b.w[0])) < 1e-11 * np.max(np.abs(b.w[0]))


def test_appended_point_on_a_vertex_has_the_vertex_column():
    lev = ogrid.Level(24, 20, 0.1, 0.0, 0.0)
    base = ib.Subdomain(lev, 6, 13, 5, 12)
    v = (3, 4)                                            # box vertex (i_lo + 3, j_lo + 4)
    x = np.array([[(base.i_lo + v[0]) * lev.h, (base.j_lo + v[1]) * lev.h]])
    sd = ib.Subdomain(lev, 6, 13, 5, 12, extra=x)
    kv = v[1] * sd.ni + v[0]
    for comp in (0, 1):
        col_v = ib.b0_column(sd, comp * sd.n_sd + kv, 100.0, 0.004)
        col_x = ib.b0_column(sd, comp * sd.n_sd + sd.n_box, 100.0, 0.004)
        assert np.max(np.abs(col_v - col_x)) < 1e-14 * np.max(np.abs(col_v))


def test_b0_with_appended_points_is_symmetric_psd():
    lev = ogrid.Level(24, 20, 0.1, 0.0, 0.0)
    extra = np.array([[1.63, 0.71], [1.71, 0.77], [0.42, 1.33]])
    sd = ib.Subdomain(lev, 6, 11, 5, 9, extra=extra)
    b = ib.b0_dense(sd, 100.0, 0.004)
    assert np.max(np.abs(b - b.T)) < 1e-14 * np.max(np.abs(b))
    assert np.min(np.linalg.eigvalsh(0.5 * (b + b.T))) > -1e-13 * np.max(np.abs(b))


def test_no_slip_at_appended_and_interpolated_points_after_corrector():
    """A moving torsional plate in the box and a stationary plate appended outside it: after the corrector
    the interpolated velocity equals the body velocities at both kinds of points."""
    w = wl.small_plate()
    ur = np.tile([0.3, -0.1], (9, 1))                       # a prescribed surface velocity on fixed points
    w["bodies"].append(dict(kind="rigid", pts=_stationary_plate(), ur=ur, appended=True))
    sim = oracle_sim(w, tol=1e-12)
    for _ in range(3):
        sim.step()
    lev = sim.levels[0]
    u, v = ogrid.faces_from_s(sim.s[0], lev)
    e0q = sim.sd.e0(u + 1.0, v)
    idx, wts = sim.last_p
    ub = np.stack([(wts * e0q[idx]).sum(1), (wts * e0q[idx + sim.sd.n_sd]).sum(1)], axis=1)
    plate, app = sim.bodies
    assert np.max(np.abs(ub[plate.n_pts:] - ur)) < 1e-10
    rx, ry = plate.r(plate.theta)
    q = plate.q()
    assert np.max(np.abs(ub[:plate.n_pts, 0] - plate.phi * q * rx)) < 1e-6
    assert np.max(np.abs(ub[:plate.n_pts, 1] - plate.phi * q * ry)) < 1e-6
