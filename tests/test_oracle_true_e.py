"""Pins of the oracle's true-E coupling (Sec. 2.2: E and E^T at the body points themselves; the operator
that Eq. operatorapprox replaces and the comparator of Sec. 5.1)."""

import numpy as np

from oracle import fsi, grid, ib


def _lev():
    return grid.Level(40, 32, 1.0 / 16, -1.0, -1.0)


def test_e_and_et_are_adjoint():
    lev = _lev()
    rng = np.random.default_rng(5)
    pts = rng.uniform([-0.4, -0.4], [0.9, 0.6], size=(7, 2))
    u = rng.standard_normal((lev.ny, lev.nx + 1))
    v = rng.standard_normal((lev.ny + 1, lev.nx))
    f = rng.standard_normal(14)
    eu, ev = ib.et_points(lev, pts, f)
    assert abs(ib.e_points(lev, pts, u, v) @ f - (np.sum(u * eu) + np.sum(v * ev))) < 1e-12


def test_e_is_exact_on_linear_velocity_fields():
    """The 3-point delta's moment conditions (sum 1, first moment 0) make E exact for linear fields at any
    point, on both staggered face families."""
    lev = _lev()
    xu, yu = lev.x0 + lev.h * np.arange(lev.nx + 1), lev.y0 + lev.h * (np.arange(lev.ny) + 0.5)
    xv, yv = lev.x0 + lev.h * (np.arange(lev.nx) + 0.5), lev.y0 + lev.h * np.arange(lev.ny + 1)
    u = 0.3 + 1.1 * xu[None, :] - 0.7 * yu[:, None]
    v = -0.2 + 0.4 * xv[None, :] + 0.9 * yv[:, None]
    pts = np.array([[0.013, -0.21], [0.5, 0.5], [-0.31, 0.377]])
    got = ib.e_points(lev, pts, u, v)
    want = np.concatenate([0.3 + 1.1 * pts[:, 0] - 0.7 * pts[:, 1], -0.2 + 0.4 * pts[:, 0] + 0.9 * pts[:, 1]])
    assert np.max(np.abs(got - want)) < 1e-13


def test_e_at_an_omega0_vertex_equals_e0_and_ke_is_symmetric_psd():
    lev = _lev()
    sd = ib.Subdomain(lev, 10, 20, 8, 18)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((lev.ny, lev.nx + 1))
    v = rng.standard_normal((lev.ny + 1, lev.nx))
    p = 3 * sd.ni + 4
    pt = np.array([[lev.x0 + sd.pi[p] * lev.h, lev.y0 + sd.pj[p] * lev.h]])
    e0 = sd.e0(u, v)
    assert np.max(np.abs(ib.e_points(lev, pt, u, v) - [e0[p], e0[sd.n_sd + p]])) < 1e-14
    pts = rng.uniform([-0.2, -0.2], [0.4, 0.3], size=(5, 2))
    ke = np.stack([ib.ke_column(lev, pts, m, 100.0, 0.004) for m in range(10)], axis=1)
    assert np.max(np.abs(ke - ke.T)) < 1e-12 * np.max(np.abs(ke))
    assert np.linalg.eigvalsh(0.5 * (ke + ke.T)).min() > -1e-12 * np.max(np.abs(ke))


def test_true_e_equals_subdomain_when_body_points_sit_on_omega0_vertices():
    """With every point on a vertex of Omega_0, P selects that vertex and P E0 = E: the sub-domain small
    system is the true one and the runs coincide."""
    h = 1.0 / 16
    pts = np.array([[0.0 + k * h, 0.125] for k in range(6)])
    runs = []
    for coupling in ("subdomain", "true"):
        body = fsi.RigidBody(pts)
        sim = fsi.Sim(40, 32, h, -1.0, -1.0, 1, 100.0, 0.004, (1.0, 0.0), (-0.5, 0.7, -0.5, 0.6), [body], h,
                      coupling=coupling)
        for _ in range(4):
            sim.step()
        runs.append(np.array([[r["bodies"][0]["fx"], r["bodies"][0]["fy"]] for r in sim.history]))
        runs.append(sim.w[0].copy())
    assert np.max(np.abs(runs[0] - runs[2])) < 1e-10 * np.max(np.abs(runs[0]))
    assert np.max(np.abs(runs[1] - runs[3])) < 1e-10 * np.max(np.abs(runs[1]))
