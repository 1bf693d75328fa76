"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test pins one oracle function to something other than itself: closed forms,
brute-force dense solves built independently here, invariants, and the values the
paper prints.  All run on the CPU.
"""

import os

import numpy as np
import pytest

from oracle import fsi, grid, ib

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- DST / solves

def test_dst_matrix_involution():
    for n in (1, 7, 31, 64):
        s = grid.dst1_matrix(n)
        assert np.allclose(s @ s, (n + 1) / 2.0 * np.eye(n), atol=1e-12 * n)


def _dense_lap(nx, ny, h):
    """-lap_h on interior vertices with zero Dirichlet ring, built entry by entry."""
    nxi, nyi = nx - 1, ny - 1
    n = nxi * nyi
    a = np.zeros((n, n))
    for j in range(nyi):
        for i in range(nxi):
            r = j * nxi + i
            a[r, r] = 4.0 / h ** 2
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < nxi and 0 <= jj < nyi:
                    a[r, jj * nxi + ii] = -1.0 / h ** 2
    return a


def test_dst_solve_matches_dense_laplacian():
    rng = np.random.default_rng(1)
    lev = grid.Level(10, 8, 0.3, 0.0, 0.0)
    rhs = rng.standard_normal((7, 9))
    got = grid.dirichlet_diag_solve(rhs, grid.lap_diag(lev))
    ref = np.linalg.solve(_dense_lap(10, 8, 0.3), rhs.ravel()).reshape(7, 9)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_aw_and_lap_solves_with_ring_values_match_dense_full_grid():
    """Dense system over ALL vertices (identity rows on the ring) vs the DST solves."""
    rng = np.random.default_rng(2)
    nx, ny, h, re, dt = 9, 7, 0.25, 40.0, 0.01
    lev = grid.Level(nx, ny, h, 0.0, 0.0)
    ring = rng.standard_normal(lev.shape)
    rhs = rng.standard_normal((ny - 1, nx - 1))
    nv = (nx + 1) * (ny + 1)

    def vid(j, i):
        return j * (nx + 1) + i

    for which in ("aw", "lap"):
        m = np.zeros((nv, nv))
        b = np.zeros(nv)
        for j in range(ny + 1):
            for i in range(nx + 1):
                r = vid(j, i)
                if i in (0, nx) or j in (0, ny):
                    m[r, r] = 1.0
                    b[r] = ring[j, i]
                    continue
                c = 1.0 / dt if which == "aw" else 0.0
                k = 1.0 / (2 * re) if which == "aw" else 1.0
                m[r, r] = c + 4.0 * k / h ** 2
                for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    m[r, vid(j + dj, i + di)] = -k / h ** 2
                b[r] = rhs[j - 1, i - 1]
        ref = np.linalg.solve(m, b).reshape(ny + 1, nx + 1)[1:-1, 1:-1]
        if which == "aw":
            got = grid.solve_aw(rhs, ring, lev, re, dt)
        else:
            got = grid.solve_lap(rhs, ring, lev)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_laplacian_inverse_exact_on_discrete_eigenmode():
    lev = grid.Level(32, 24, 1.0 / 32, 0.0, 0.0)
    x, y = lev.xv(), lev.yv()
    k, l = 3, 5
    lx, ly = 1.0, 24.0 / 32
    s = np.sin(k * np.pi * x[None, :] / lx) * np.sin(l * np.pi * y[:, None] / ly)
    lam = (4 / lev.h ** 2) * (np.sin(np.pi * k / (2 * 32)) ** 2 + np.sin(np.pi * l / (2 * 24)) ** 2)
    got = grid.solve_lap(lam * s[1:-1, 1:-1], np.zeros(lev.shape), lev)
    assert np.max(np.abs(got - s[1:-1, 1:-1])) < 1e-13


def test_laplacian_inverse_second_order_on_smooth_solution():
    errs = []
    for n in (16, 32, 64):
        lev = grid.Level(n, n, 1.0 / n, 0.0, 0.0)
        x, y = np.meshgrid(lev.xv(), lev.yv())
        s = np.exp(x) * np.sin(np.pi * x) * np.sin(np.pi * y)
        w = np.exp(x) * np.sin(np.pi * y) * ((2 * np.pi ** 2 - 1) * np.sin(np.pi * x) - 2 * np.pi * np.cos(np.pi * x))
        got = grid.solve_lap(w[1:-1, 1:-1], np.zeros(lev.shape), lev)
        errs.append(np.max(np.abs(got - s[1:-1, 1:-1])))
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4


def test_paper_condition_number_of_viscous_operator():
    """Sec. 3.2.1: alpha = 0.125 (Re dx = 1, dt = dx/4) gives cond(I + alpha Lambda) = 2."""
    vals = dict(l.split() for l in open(os.path.join(GOLDEN, "paper_condition_number.txt")) if l[0] != "#")
    n, h = 512, 1.0 / 512
    re, dt = 1.0 / h, h / 4.0
    assert abs(dt / (2 * re * h * h) - float(vals["alpha"])) < 1e-15
    d = grid.aw_diag(grid.Level(n, n, h, 0.0, 0.0), re, dt)
    assert abs(d.max() / d.min() - float(vals["condition_number"])) < 1e-4


# --------------------------------------------------------------------------- C, curl, N

def test_curl_of_velocity_is_minus_laplacian():
    rng = np.random.default_rng(3)
    lev = grid.Level(11, 9, 0.2, 0.0, 0.0)
    s = rng.standard_normal(lev.shape)
    u, v = grid.faces_from_s(s, lev)
    assert np.allclose(grid.curl_faces(u, v, lev), -grid.laplacian(s, lev), atol=1e-10)


def test_velocity_faces_from_streamfunction_of_uniform_flow():
    lev = grid.Level(6, 5, 0.5, -1.0, 2.0)
    x, y = np.meshgrid(lev.xv(), lev.yv())
    u, v = grid.faces_from_s(2.0 * y - 3.0 * x, lev)    # s = U y - V x  ->  (u, v) = (U, V)
    assert np.allclose(u, 2.0) and np.allclose(v, 3.0)


def test_nonlinear_term_uniform_freestream_is_central_difference():
    rng = np.random.default_rng(4)
    lev = grid.Level(10, 8, 0.1, 0.0, 0.0)
    w = np.zeros(lev.shape)
    w[1:-1, 1:-1] = rng.standard_normal((7, 9))
    n = grid.nonlinear(np.zeros(lev.shape), w, lev, (1.5, -0.5))
    ref = 1.5 * (w[1:-1, 2:] - w[1:-1, :-2]) / 0.2 - 0.5 * (w[2:, 1:-1] - w[:-2, 1:-1]) / 0.2
    assert np.allclose(n, ref, atol=1e-12)


def test_nonlinear_term_shear_flows_use_vertex_averaged_velocity():
    rng = np.random.default_rng(5)
    lev = grid.Level(10, 8, 0.1, 0.0, 0.0)
    w = rng.standard_normal(lev.shape)
    sy = rng.standard_normal(lev.ny + 1)                  # s(y): u = u(y), v = 0
    s = np.repeat(sy[:, None], lev.nx + 1, axis=1)
    n = grid.nonlinear(s, w, lev, (0.0, 0.0))
    uface = (sy[1:] - sy[:-1]) / lev.h                     # u at y_{j+1/2}
    ubar = 0.5 * (uface[1:] + uface[:-1])                  # at y_j, j = 1..ny-1
    ref = ubar[:, None] * (w[1:-1, 2:] - w[1:-1, :-2]) / (2 * lev.h)
    assert np.allclose(n, ref, atol=1e-10)
    sx = rng.standard_normal(lev.nx + 1)                  # s(x): v = v(x), u = 0
    s = np.repeat(sx[None, :], lev.ny + 1, axis=0)
    n = grid.nonlinear(s, w, lev, (0.0, 0.0))
    vface = -(sx[1:] - sx[:-1]) / lev.h
    vbar = 0.5 * (vface[1:] + vface[:-1])
    ref = vbar[None, :] * (w[2:, 1:-1] - w[:-2, 1:-1]) / (2 * lev.h)
    assert np.allclose(n, ref, atol=1e-10)


def test_crank_nicolson_decay_of_small_eigenmode():
    """No body, U_inf = 0: a tiny discrete eigenmode decays by the CN factor each step."""
    nx, ny, h, re, dt = 32, 32, 1.0 / 32, 50.0, 0.01
    sim = fsi.Sim(nx, ny, h, 0.0, 0.0, 1, re, dt, (0.0, 0.0), None, [], h)
    lev = sim.levels[0]
    x, y = np.meshgrid(lev.xv(), lev.yv())
    k, l = 2, 3
    lam = (4 / h ** 2) * (np.sin(np.pi * k / 64) ** 2 + np.sin(np.pi * l / 64) ** 2)
    eps = 1e-9
    w0 = eps * np.sin(k * np.pi * x) * np.sin(l * np.pi * y)
    sim.w[0][:] = w0
    sim.s[0][:] = w0 / lam
    g = (1 / dt - lam / (2 * re)) / (1 / dt + lam / (2 * re))
    for n in range(1, 6):
        sim.step()
        assert np.max(np.abs(sim.w[0] - g ** n * w0)) < 1e-6 * eps


# --------------------------------------------------------------------------- delta, E0, P

def test_delta_moment_conditions():
    rng = np.random.default_rng(6)
    j = np.arange(-4, 5)
    for r in rng.uniform(-1, 1, 50):
        phi = ib.delta3(r - j)
        assert abs(phi.sum() - 1.0) < 1e-14
        assert abs(((r - j) * phi).sum()) < 1e-14
        assert abs((phi ** 2).sum() - 0.5) < 1e-14


def test_e0_weights_at_vertices():
    lev = grid.Level(16, 16, 0.1, 0.0, 0.0)
    sd = ib.Subdomain(lev, 4, 6, 5, 7)
    _, _, w = sd._u_window()
    ref = np.outer([0, 0.5, 0.5, 0], [0, 1 / 6, 2 / 3, 1 / 6, 0])
    assert np.allclose(w[0], ref, atol=1e-15)
    _, _, w = sd._v_window()
    assert np.allclose(w[0], ref.T, atol=1e-15)


def test_e0_adjointness_and_partition_of_unity():
    rng = np.random.default_rng(7)
    lev = grid.Level(20, 18, 0.1, 0.0, 0.0)
    sd = ib.Subdomain(lev, 3, 12, 4, 14)
    u = rng.standard_normal((lev.ny, lev.nx + 1))
    v = rng.standard_normal((lev.ny + 1, lev.nx))
    g = rng.standard_normal(2 * sd.n_sd)
    eu, ev = sd.e0t(g)
    assert abs(sd.e0(u, v) @ g - (np.sum(u * eu) + np.sum(v * ev))) < 1e-12
    e = sd.e0(np.full_like(u, 2.0), np.full_like(v, -1.0))
    assert np.allclose(e[: sd.n_sd], 2.0) and np.allclose(e[sd.n_sd:], -1.0)


def test_hat_interpolation_rows():
    rng = np.random.default_rng(8)
    lev = grid.Level(20, 20, 0.1, -1.0, -1.0)
    sd = ib.Subdomain(lev, 3, 15, 2, 17)
    pts = np.stack([rng.uniform(-0.7, 0.5, 40), rng.uniform(-0.8, 0.7, 40)], axis=1)
    pts[0] = (lev.x0 + 15 * lev.h, lev.y0 + 17 * lev.h)   # corner of the box (clamped cell)
    idx, wts = sd.p_rows(pts)
    assert np.allclose(wts.sum(axis=1), 1.0)
    xs = lev.x0 + sd.pi * lev.h
    ys = lev.y0 + sd.pj * lev.h
    lin = 0.3 + 1.7 * xs - 0.9 * ys                     # the hat reproduces linear functions
    assert np.allclose((wts * lin[idx]).sum(axis=1), 0.3 + 1.7 * pts[:, 0] - 0.9 * pts[:, 1])
    assert np.allclose(ib.hat([0.0, 0.05, 0.1, -0.05], 0.1), [1.0, 0.5, 0.0, 0.5])
    with pytest.raises(ValueError):
        sd.p_rows(np.array([[0.9, 0.0]]))


# --------------------------------------------------------------------------- B0

def _dense_ops(nx, ny, h, sd, re, dt):
    """Dense C, A_q = I/dt + C C^T/(2 Re) (Sec. 3.2.1) and E0, built independently."""
    nxi, nyi = nx - 1, ny - 1
    ns = nxi * nyi
    nu, nv = ny * (nx + 1), (ny + 1) * nx

    def sid(j, i):
        return (j - 1) * nxi + (i - 1) if (1 <= i <= nxi and 1 <= j <= nyi) else None

    c = np.zeros((nu + nv, ns))
    for j in range(ny):
        for i in range(nx + 1):
            r = j * (nx + 1) + i
            for jj, sg in ((j + 1, 1.0), (j, -1.0)):
                k = sid(jj, i)
                if k is not None:
                    c[r, k] += sg / h
    for j in range(ny + 1):
        for i in range(nx):
            r = nu + j * nx + i
            for ii, sg in ((i + 1, -1.0), (i, 1.0)):
                k = sid(j, ii)
                if k is not None:
                    c[r, k] += sg / h
    aq = np.eye(nu + nv) / dt + c @ c.T / (2 * re)
    e0 = np.zeros((2 * sd.n_sd, nu + nv))
    xu = np.arange(nx + 1) * h
    yu = (np.arange(ny) + 0.5) * h
    xv = (np.arange(nx) + 0.5) * h
    yv = np.arange(ny + 1) * h
    for p in range(sd.n_sd):
        px, py = sd.pi[p] * h, sd.pj[p] * h
        e0[p, :nu] = np.outer(ib.delta3((yu - py) / h), ib.delta3((xu - px) / h)).ravel()
        e0[sd.n_sd + p, nu:] = np.outer(ib.delta3((yv - py) / h), ib.delta3((xv - px) / h)).ravel()
    return c, aq, e0


def test_b0_columns_match_dense_brute_force():
    nx, ny, h, re, dt = 14, 12, 0.125, 80.0, 0.01
    lev = grid.Level(nx, ny, h, 0.0, 0.0)
    sd = ib.Subdomain(lev, 4, 7, 3, 6)
    b0 = ib.b0_dense(sd, re, dt)
    c, aq, e0 = _dense_ops(nx, ny, h, sd, re, dt)
    ref = e0 @ c @ np.linalg.solve(c.T @ aq @ c, c.T @ e0.T)
    assert np.max(np.abs(b0 - ref)) < 1e-12 * np.max(np.abs(ref))


def test_b0_symmetric_positive_semidefinite():
    lev = grid.Level(24, 20, 0.1, 0.0, 0.0)
    sd = ib.Subdomain(lev, 6, 11, 5, 10)
    b0 = ib.b0_dense(sd, 100.0, 0.004)
    scale = np.max(np.abs(b0))
    assert np.max(np.abs(b0 - b0.T)) < 1e-14 * scale * 10
    ev = np.linalg.eigvalsh(0.5 * (b0 + b0.T))
    assert ev.min() > -1e-13 * scale


# --------------------------------------------------------------------------- structure / FSI

def test_newmark_torsion_conserves_energy_and_has_trapezoid_period():
    dt, i, k, th0 = 0.05, 1.3, 0.7, 0.4
    b = fsi.TorsionalBody((0, 0), 0.0, 2, 0.1, i, 0.0, k, th0)
    om = np.sqrt(k / i)
    omd = 2.0 * np.arctan(om * dt / 2.0) / dt
    e0 = i * b.phi ** 2 + k * b.theta ** 2
    for n in range(1, 200):
        r_phi, r_theta = b.rhs_terms(dt)
        b.advance(r_phi / b.jac(dt), r_theta, dt)          # f = 0: theta = J^{-1} r^phi
        assert abs(i * b.phi ** 2 + k * b.theta ** 2 - e0) < 1e-12
        assert abs(b.theta - th0 * np.cos(omd * n * dt)) < 1e-12


def _small_case(stiff=0.5, inertia=1.0, theta=np.deg2rad(20), theta0=0.0, n_pts=9, **kw):
    h = 1.0 / 16
    body = fsi.TorsionalBody((0.0, 0.0), theta0, n_pts, h, inertia, 0.0, stiff, theta)
    sim = fsi.Sim(48, 40, h, -1.0, -1.25, 1, 100.0, 0.004, (1.0, 0.0), (-0.6, 0.8, -0.7, 0.8), [body], h, **kw)
    return sim, body


def _advance(sim, n):
    for _ in range(n):
        sim.step()


def test_block_lu_iterate_matches_dense_coupled_system():
    """One FSI iteration (Eqs. stress2, dtheta2, corrector2) equals the dense solve of the
    linearised block system of App. A (Eq. bigsystem) with E -> P E0."""
    sim, body = _small_case(inertia=0.05, tol=1e30)
    _advance(sim, 3)
    dt, ds, lev, sd = sim.dt, sim.ds, sim.levels[0], sim.sd
    sim._r_phi, sim._r_theta = {}, {}
    r_phi, r_theta = body.rhs_terms(dt)
    sim._r_phi[id(body)], sim._r_theta[id(body)] = r_phi, r_theta
    th0, ph0 = body.theta, body.phi
    sim.predictor()
    s_star = sim.s[0][1:-1, 1:-1].ravel().copy()
    f, theta_k, _, _ = sim.fsi()
    sim.corrector(f)
    s_new = sim.s[0][1:-1, 1:-1].ravel()

    c, aq, e0 = _dense_ops(lev.nx, lev.ny, lev.h, sd, sim.re, dt)
    nb = body.n_pts
    idx, wts = sd.p_rows(body.points(th0))
    p = np.zeros((2 * nb, 2 * sd.n_sd))
    for q in range(nb):
        for k in range(4):
            p[q, idx[q, k]] += wts[q, k]
            p[nb + q, sd.n_sd + idx[q, k]] += wts[q, k]
    e = p @ e0
    rx, ry = body.r(th0)
    sv = np.concatenate([body.q() * rx, body.q() * ry])
    jac = body.jac(dt)
    nu = lev.ny * (lev.nx + 1)
    qinf = np.concatenate([np.full(nu, 1.0), np.zeros(c.shape[0] - nu)])
    ns, nf = c.shape[1], 2 * nb
    n = ns + 2 + nf
    m = np.zeros((n, n))
    rhs = np.zeros(n)
    cac = c.T @ aq @ c
    m[:ns, :ns] = cac
    m[:ns, ns + 2:] = (ds / lev.h ** 2) * c.T @ e.T
    rhs[:ns] = cac @ s_star
    m[ns, ns + 1] = jac                              # J dtheta - ds S f = r^phi - J theta^(k)
    m[ns, ns + 2:] = -ds * sv
    rhs[ns] = r_phi - jac * th0
    m[ns + 1, ns] = -1.0                             # -dphi + (2/dt) dtheta = r^theta - (2/dt) theta + phi
    m[ns + 1, ns + 1] = 2.0 / dt
    rhs[ns + 1] = r_theta - 2.0 / dt * th0 + ph0
    m[ns + 2:, :ns] = e @ c                          # E C s - S^T dphi = -E q_inf + S^T phi^(k)
    m[ns + 2:, ns] = -sv
    rhs[ns + 2:] = -e @ qinf + sv * ph0
    sol = np.linalg.solve(m, rhs)
    assert np.max(np.abs(sol[ns + 2:] - f)) < 1e-9 * np.max(np.abs(f))
    assert abs(sol[ns + 1] - (theta_k[id(body)] - th0)) < 1e-12 + 1e-9 * abs(sol[ns + 1])
    assert np.max(np.abs(sol[:ns] - s_new)) < 1e-10 * np.max(np.abs(s_new))


def test_no_slip_holds_after_corrector():
    sim, body = _small_case()
    _advance(sim, 4)
    lev, sd, nb = sim.levels[0], sim.sd, sim.nb
    u, v = grid.faces_from_s(sim.s[0], lev)
    e0q = sd.e0(u + 1.0, v)
    idx, wts = sim.last_p
    ub = np.concatenate([(wts * e0q[idx]).sum(1), (wts * e0q[idx + sd.n_sd]).sum(1)])
    target = sim.last_svec[id(body)] * body.phi
    assert np.max(np.abs(ub - target)) < 1e-10 * max(1.0, np.max(np.abs(ub)))


def test_stiff_spring_limit_matches_stationary_plate():
    th = np.deg2rad(20)
    diffs = []
    for k in (1e6, 1e8):
        sim_t, body = _small_case(stiff=k, inertia=1e-3, theta=0.0, theta0=th)
        _advance(sim_t, 5)
        pts = body.points(0.0)
        h = sim_t.ds
        rigid = fsi.RigidBody(fsi.TorsionalBody((0, 0), th, body.n_pts, h, 1, 0, 1, 0).points(0.0))
        sim_r = fsi.Sim(48, 40, h, -1.0, -1.25, 1, 100.0, 0.004, (1.0, 0.0), (-0.6, 0.8, -0.7, 0.8), [rigid], h)
        _advance(sim_r, 5)
        ft = np.array([[r["bodies"][0]["fx"], r["bodies"][0]["fy"]] for r in sim_t.history])
        fr = np.array([[r["bodies"][0]["fx"], r["bodies"][0]["fy"]] for r in sim_r.history])
        diffs.append(np.max(np.abs(ft - fr)) / np.max(np.abs(fr)))
        assert np.allclose(pts, rigid.pts, atol=1e-15)
    assert diffs[1] < 1e-3
    assert 50 < diffs[0] / diffs[1] < 200            # differences scale as O(1/k)


def test_fsi_iteration_contracts_within_three_iterations():
    sim, _ = _small_case()
    _advance(sim, 6)
    assert all(1 <= r["iters"] <= 3 for r in sim.history)


def test_multidomain_coupling_exact_for_coincident_and_linear_fields():
    levs = grid.make_levels(16, 12, 0.1, -0.5, -0.3, 2)
    fine, coarse = levs
    xc, yc = np.meshgrid(coarse.xv(), coarse.yv())
    lin = 0.2 + 1.3 * xc - 0.7 * yc
    ff = np.zeros(fine.shape)
    grid.set_ring_from_coarse(ff, fine, lin, coarse)
    xf, yf = np.meshgrid(fine.xv(), fine.yv())
    ref = 0.2 + 1.3 * xf - 0.7 * yf
    ring = np.ones(fine.shape, bool)
    ring[1:-1, 1:-1] = False
    assert np.allclose(ff[ring], ref[ring], atol=1e-13)
    wc = np.zeros(coarse.shape)
    wf = np.cos(xf) * np.sin(3 * yf)
    grid.inject_fine_to_coarse(wf, fine, wc, coarse)
    inside = (xc > fine.xv()[0]) & (xc < fine.xv()[-1]) & (yc > fine.yv()[0]) & (yc < fine.yv()[-1])
    assert np.allclose(wc[inside], (np.cos(xc) * np.sin(3 * yc))[inside], atol=1e-14)
    assert np.all(wc[~inside] == 0)
