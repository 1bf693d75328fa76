"""Pins of the oracle's deformable body (Sec. 2.1 Eq. beam, App. A; corotational beam of reading R18)
against mechanics that does not come from the oracle: energy gradients, frame invariance, the cubic
cantilever solution, the elastica, the cantilever's characteristic equation, Newmark energy
conservation, and a dense solve of the linearised coupled system."""

import numpy as np
import pytest

from oracle import beam, fsi, grid
from tests.test_oracle_pins import _dense_ops

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _static(bm, load, steps=1, max_it=40):
    """Newton solve of R(chi) = load (a nodal load vector over the free dofs), load applied in steps;
    returns chi and the max-norm of every Newton increment of the last load step."""
    chi = bm.chi.copy()
    inc = []
    for s in range(1, steps + 1):
        fext = load * s / steps
        inc = []
        for _ in range(max_it):
            r, k = bm.internal(chi)
            d = np.linalg.solve(k, fext - r)
            chi = chi + d
            inc.append(np.max(np.abs(d)))
            if inc[-1] < 1e-13:
                break
    return chi, inc


def test_tangent_is_derivative_of_internal_force_and_force_is_energy_gradient():
    rng = np.random.default_rng(3)
    bm = beam.Beam((0.2, -0.1), 0.3, 6, 0.2, 0.1, 1e-3, 1e3, tip_angle=0.8)
    chi = bm.chi + 1e-3 * rng.standard_normal(bm.ndof)
    r, k = bm.internal(chi)
    e = 1e-6
    kfd = np.zeros_like(k)
    g = np.zeros(bm.ndof)
    zero = np.zeros(bm.ndof)
    for j in range(bm.ndof):
        d = np.zeros(bm.ndof)
        d[j] = e
        kfd[:, j] = (bm.internal(chi + d)[0] - bm.internal(chi - d)[0]) / (2 * e)
        g[j] = (bm.energy(chi + d, zero) - bm.energy(chi - d, zero)) / (2 * e)
    assert np.max(np.abs(k - kfd)) < 1e-8 * np.max(np.abs(k))
    assert np.max(np.abs(k - k.T)) < 1e-12 * np.max(np.abs(k))
    assert np.max(np.abs(r - g)) < 1e-7 * np.max(np.abs(r))


def test_element_is_frame_invariant():
    bm = beam.Beam((0, 0), 0.0, 2, 0.5, 1.0, 2.0, 50.0)
    pa, pb = np.array([0.1, 0.2, 0.05]), np.array([0.55, 0.35, -0.1])
    f, k = bm.element(pa, pb)
    for a in (0.7, -2.1):
        c, s = np.cos(a), np.sin(a)
        q = np.array([[c, -s], [s, c]])
        t = np.array([1.3, -0.4])
        # rigid motion of the undeformed element: no force
        fa, _ = bm.element(np.array([*t, a]), np.array([*(t + q @ [0.5, 0.0]), a]))
        assert np.max(np.abs(fa)) < 1e-12
        # a rotated deformed element: forces rotate with it, moments unchanged
        fr, _ = bm.element(np.array([*(q @ pa[:2] + t), pa[2] + a]), np.array([*(q @ pb[:2] + t), pb[2] + a]))
        assert np.allclose(fr[0:2], q @ f[0:2], atol=1e-12)
        assert np.allclose(fr[3:5], q @ f[3:5], atol=1e-12)
        assert np.allclose(fr[[2, 5]], f[[2, 5]], atol=1e-12)
    # equilibrium of one element: forces sum to zero, moments about node a sum to zero
    assert abs(f[0] + f[3]) < 1e-12 and abs(f[1] + f[4]) < 1e-12
    mom = f[2] + f[5] + (pb[0] - pa[0]) * f[4] - (pb[1] - pa[1]) * f[3]
    assert abs(mom) < 1e-12


def test_small_tip_load_gives_cubic_cantilever_solution():
    """Linear theory: tip deflection P L^3 / (3 EI) and tip slope P L^2 / (2 EI), nodally exact for
    cubic elements; the nonlinear beam agrees up to O((P L^2 / EI)^2)."""
    for alpha in (0.0, 0.6):
        bm = beam.Beam((0, 0), alpha, 10, 0.1, 1.0, 2.0, 1e6)
        p = 2e-3
        load = np.zeros(bm.ndof)
        load[-3:-1] = p * np.array([-np.sin(alpha), np.cos(alpha)])
        chi, _ = _static(bm, load)
        tip, _ = bm.tip_deflection(chi, np.zeros(bm.ndof))
        assert abs(tip - p / (3 * 2.0)) < 1e-6 * p / 6.0
        assert abs(chi[-1] - p / (2 * 2.0)) < 1e-6 * p / 4.0
        # every node: w(s) = P s^2 (3 L - s) / (6 EI)
        s = np.arange(1, 11) * 0.1
        w = (chi.reshape(10, 3)[:, :2] - bm.x0[1:]) @ np.array([-np.sin(alpha), np.cos(alpha)])
        assert np.max(np.abs(w - p * s ** 2 * (3 - s) / 12.0)) < 1e-6 * p


def _elastica(k):
    """Tip of a cantilever under a transverse dead tip load with k = P L^2 / EI, by shooting on the
    elastica theta'' = -k cos(theta), theta(0) = 0, theta'(1) = 0."""
    from scipy.integrate import solve_ivp
    from scipy.optimize import brentq

    def end(c):
        sol = solve_ivp(lambda s, y: [y[1], -k * np.cos(y[0]), np.cos(y[0]), np.sin(y[0])], [0, 1],
                        [0, c, 0, 0], rtol=1e-12, atol=1e-14)
        return sol.y[:, -1]
    c0 = brentq(lambda c: end(c)[1], 1e-3, 5 * k)
    th, _, x, y = end(c0)
    return y, 1 - x, th


def test_large_tip_load_converges_to_elastica_and_newton_is_quadratic():
    pytest.importorskip("scipy")
    v_ref, u_ref, th_ref = _elastica(1.0)
    errs = []
    for n in (10, 20, 40):
        bm = beam.Beam((0, 0), 0.0, n, 1.0 / n, 1.0, 1.0, 1e6)      # axial strain P/EA = 1e-6
        load = np.zeros(bm.ndof)
        load[-2] = 1.0
        chi, inc = _static(bm, load, steps=4)
        errs.append(max(abs(chi[-2] - v_ref) / v_ref, abs(1 - chi[-3] - u_ref) / u_ref, abs(chi[-1] - th_ref) / th_ref))
        # quadratic convergence of the Newton iteration (consistent tangent): the last increment above
        # round-off is followed by one of the order of its square, in few iterations
        assert len(inc) <= 8 and inc[-1] < 1e-13
        big = [x for x in inc if x > 1e-12]
        assert inc[len(big)] < 10.0 * big[-1] ** 2 and big[-1] < 1e-5
    assert errs[-1] < 2e-4
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5   # second order in ds


def test_cantilever_first_frequency_from_characteristic_equation():
    """omega_1 = beta_1^2 sqrt(EI / mu) / L^2, beta_1 the first root of cos(b) cosh(b) = -1."""
    from scipy.linalg import eigh
    from scipy.optimize import brentq
    b1 = brentq(lambda b: np.cos(b) * np.cosh(b) + 1.0, 1.5, 2.5)
    mu, ei, length = 0.1, 1e-3, 1.0
    om = b1 ** 2 * np.sqrt(ei / mu) / length ** 2
    errs = []
    for n in (25, 50):
        bm = beam.Beam((0, 0), 0.0, n, length / n, mu, ei, 1e3)
        _, k = bm.internal(bm.chi)
        ev = eigh(k, np.diag(bm.mass()), eigvals_only=True)
        errs.append(abs(np.sqrt(ev[0]) - om) / om)
    assert errs[1] < 5e-4
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_newmark_free_vibration_conserves_energy_at_small_amplitude():
    """Trapezoidal Newmark without load conserves kinetic + strain energy exactly for a linear system;
    at small amplitude the beam is linear up to O(amplitude^2)."""
    dt = 0.05
    for amp, tol in ((1e-4, 1e-7), (1e-2, 1e-3)):
        bm = beam.Beam((0, 0), 0.2, 10, 0.1, 0.1, 1e-3, 1e3, tip_angle=amp)
        e0 = bm.energy()
        m = bm.mass()
        for _ in range(120):
            r_zeta, r_chi = bm.rhs_terms(dt)
            chi = bm.chi.copy()
            for _ in range(30):                      # (4/dt^2) M chi + R(chi) = r^zeta
                r, k = bm.internal(chi)
                g = 4.0 / dt ** 2 * m * chi + r - r_zeta
                if np.max(np.abs(g)) < 1e-15 * np.max(np.abs(r_zeta)):
                    break
                chi = chi - np.linalg.solve(np.diag(4.0 / dt ** 2 * m) + k, g)
            bm.advance(chi, r_chi, dt)
        assert abs(bm.energy() - e0) < tol * e0


# --------------------------------------------------------------------------- FSI with the flag

def _flag_case(ei=1e-3, ea=1e3, mu=0.1, tip=0.1, n_el=8, **kw):
    h = 1.0 / 16
    bm = beam.Beam((0.0, 0.0), 0.0, n_el, h, mu, ei, ea, tip_angle=tip)
    sim = fsi.Sim(48, 40, h, -1.0, -1.25, 1, 100.0, 0.004, (1.0, 0.0), (-0.6, 0.8, -0.7, 0.8), [bm], h, **kw)
    return sim, bm


def test_flag_iterate_matches_dense_coupled_system():
    """One FSI iteration for the flag (Eqs. stress2 and dchi2 with J_d = 4 M/dt^2 + K(chi)) equals the
    dense solve of the linearised block system: fluid, Newmark beam, no-slip at the nodes."""
    sim, bm = _flag_case(tol=1e30)
    for _ in range(3):
        sim.step()
    dt, ds, lev, sd = sim.dt, sim.ds, sim.levels[0], sim.sd
    r_zeta, r_chi = bm.rhs_terms(dt)
    sim._r_phi, sim._r_theta = {id(bm): r_zeta}, {id(bm): r_chi}
    chi0 = bm.chi.copy()
    sim.predictor()
    s_star = sim.s[0][1:-1, 1:-1].ravel().copy()
    f, chi_k, _, _ = sim.fsi()
    sim.corrector(f)
    s_new = sim.s[0][1:-1, 1:-1].ravel()

    c, aq, e0 = _dense_ops(lev.nx, lev.ny, lev.h, sd, sim.re, dt)
    nb, nd = bm.n_pts, bm.ndof
    idx, wts = sd.p_rows(bm.points(chi0))
    p = np.zeros((2 * nb, 2 * sd.n_sd))
    for q in range(nb):
        for k in range(4):
            p[q, idx[q, k]] += wts[q, k]
            p[nb + q, sd.n_sd + idx[q, k]] += wts[q, k]
    e = p @ e0
    # node q >= 1 translations are dofs 3(q-1), 3(q-1)+1 (the clamp, node 0, has none)
    t = np.zeros((2 * nb, nd))
    for q in range(1, nb):
        t[q, 3 * (q - 1)] = 1.0
        t[nb + q, 3 * (q - 1) + 1] = 1.0
    rint, kt = bm.internal(chi0)
    m = bm.mass()
    jd = np.diag(4.0 / dt ** 2 * m) + kt
    nu = lev.ny * (lev.nx + 1)
    qinf = np.concatenate([np.full(nu, 1.0), np.zeros(c.shape[0] - nu)])
    ns, nf = c.shape[1], 2 * nb
    n = ns + nd + nf
    a = np.zeros((n, n))
    rhs = np.zeros(n)
    cac = c.T @ aq @ c
    a[:ns, :ns] = cac
    a[:ns, ns + nd:] = (ds / lev.h ** 2) * c.T @ e.T
    rhs[:ns] = cac @ s_star
    a[ns:ns + nd, ns:ns + nd] = jd                   # J dchi - ds T^T f = r^zeta - (4/dt^2) M chi - R(chi)
    a[ns:ns + nd, ns + nd:] = -ds * t.T
    rhs[ns:ns + nd] = r_zeta - 4.0 / dt ** 2 * m * chi0 - rint
    a[ns + nd:, :ns] = e @ c                         # E C s - (2/dt) T dchi = -E q_inf + T((2/dt) chi - r^chi)
    a[ns + nd:, ns:ns + nd] = -2.0 / dt * t
    rhs[ns + nd:] = -e @ qinf + t @ (2.0 / dt * chi0 - r_chi)
    sol = np.linalg.solve(a, rhs)
    assert np.max(np.abs(sol[ns + nd:] - f)) < 1e-9 * np.max(np.abs(f))
    dchi = chi_k[id(bm)] - chi0
    assert np.max(np.abs(sol[ns:ns + nd] - dchi)) < 1e-9 * np.max(np.abs(dchi))
    assert np.max(np.abs(sol[:ns] - s_new)) < 1e-10 * np.max(np.abs(s_new))


def test_flag_no_slip_holds_after_corrector():
    sim, bm = _flag_case()
    for _ in range(4):
        sim.step()
    lev, sd, nb = sim.levels[0], sim.sd, sim.nb
    u, v = grid.faces_from_s(sim.s[0], lev)
    e0q = sd.e0(u + 1.0, v)
    idx, wts = sim.last_p
    ub = np.concatenate([(wts * e0q[idx]).sum(1), (wts * e0q[idx + sd.n_sd]).sum(1)])
    vel = np.zeros((nb, 2))
    vel[1:] = bm.zeta.reshape(-1, 3)[:, :2]
    target = np.concatenate([vel[:, 0], vel[:, 1]])
    # P at the last iterate's points, velocities T zeta_{n+1} of the converged state (Eq. corrector2)
    assert np.max(np.abs(ub - target)) < 1e-10 * max(1.0, np.max(np.abs(ub)))


def test_stiff_flag_limit_matches_stationary_plate():
    diffs = []
    for ei in (1e2, 1e4):
        sim_f, bm = _flag_case(ei=ei, ea=1e3 * ei, tip=0.0)
        for _ in range(4):
            sim_f.step()
        rigid = fsi.RigidBody(bm.x0)
        sim_r = fsi.Sim(48, 40, sim_f.ds, -1.0, -1.25, 1, 100.0, 0.004, (1.0, 0.0), (-0.6, 0.8, -0.7, 0.8),
                        [rigid], sim_f.ds)
        for _ in range(4):
            sim_r.step()
        ff = np.array([[r["bodies"][0]["fx"], r["bodies"][0]["fy"]] for r in sim_f.history])
        fr = np.array([[r["bodies"][0]["fx"], r["bodies"][0]["fy"]] for r in sim_r.history])
        diffs.append(np.max(np.abs(ff - fr)) / np.max(np.abs(fr)))
    assert diffs[1] < 1e-3
    assert 30 < diffs[0] / diffs[1] < 300            # differences scale as O(1/EI)


def test_flag_fsi_iteration_contracts_linearly():
    sim, _ = _flag_case(tip=0.3)
    for _ in range(6):
        sim.step()
    assert all(2 <= r["iters"] <= 5 for r in sim.history)
