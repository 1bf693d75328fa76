"""Pins of the oracle's prescribed flapping kinematics and hinged passive plate (Sec. 5.1, Eq. newtonseldg,
reading R20) against closed forms, finite differences, a Lagrangian derivation and limiting cases."""

import numpy as np
import pytest

from oracle import fsi as ofsi
from oracle import grid as ogrid
from oracle import kinematics as okin
from paper_2103_06415_gb300 import workloads as wl

from runners import oracle_history, oracle_sim


def _fd(fun, t, h=1e-4):
    """Five-point first derivative."""
    return (-fun(t + 2 * h) + 8 * fun(t + h) - 8 * fun(t - h) + fun(t - 2 * h)) / (12 * h)


@pytest.mark.parametrize("sigma", [3.770, 0.628])
def test_kinematic_derivatives_match_finite_differences(sigma):
    kin = okin.FlappingKinematics(1.4, np.pi / 4, sigma, sigma, freq=1.3)
    for t in (0.05, 0.21, 0.4, 0.77, 1.6):
        s = kin.state(t)
        for k, kd in ((0, 1), (1, 2), (3, 4), (4, 5)):
            fd = _fd(lambda u: kin.state(u)[k], t)
            assert abs(fd - s[kd]) < 1e-7 * max(1.0, abs(s[kd])), (t, k)


def test_kinematics_initial_values_and_periodic_shape_function():
    kin = okin.FlappingKinematics(1.4, np.pi / 4, 3.77, 3.77)
    x, xd, _, a, ad, _ = kin.state(0.0)
    assert x == 0.0 and xd == 0.0                 # start-up conditioner: no impulsive heave
    assert abs(a + np.pi / 4) < 1e-15 and ad == 0.0
    assert abs(kin.g_t(0.5)) < 1e-13              # tanh(sigma cos) is odd about tau = 1/4
    assert abs(kin.g_t(1.3) - kin.g_t(0.3)) < 1e-13
    assert all(kin.g_t(t) <= kin.gt_max + 1e-15 for t in np.linspace(0, 1, 41))


def test_small_sigma_reduces_to_harmonic_kinematics():
    """sigma -> 0: G_t / max G_t -> sin(2 pi tau), G_r / max G_r -> cos(2 pi tau)."""
    sig = 1e-3
    kin = okin.FlappingKinematics(1.4, np.pi / 4, sig, sig)
    for t in (0.1, 0.37, 0.8, 2.2):
        x, _, _, a, _, _ = kin.state(t)
        c0 = (np.tanh(8 * t - 2) + np.tanh(2)) / (1 + np.tanh(2))
        assert abs(x - 0.7 * np.sin(2 * np.pi * t) * c0) < 1e-6
        assert abs(a + np.pi / 4 * np.cos(2 * np.pi * t)) < 1e-6


def test_pseudo_moment_matches_lagrangian_of_hinged_plate():
    """g of Eq. newtonseldg against Lagrange's equation for a rigid plate (mass m, centre of mass l2 from the
    hinge, inertia I about the hinge) whose hinge rides at l1 along a plate with prescribed X1(t), alpha1(t)."""
    sp = pytest.importorskip("sympy")
    t = sp.symbols("t")
    m, l1, l2, inert = sp.symbols("m l1 l2 I", positive=True)
    X, al, th = sp.Function("X")(t), sp.Function("al")(t), sp.Function("th")(t)
    hinge = sp.Matrix([X + l1 * sp.sin(al), -l1 * sp.cos(al)])
    phi = al + th
    cg = hinge + l2 * sp.Matrix([sp.sin(phi), -sp.cos(phi)])
    v = cg.diff(t)
    kinetic = sp.Rational(1, 2) * m * (v.T * v)[0] + sp.Rational(1, 2) * (inert - m * l2 ** 2) * phi.diff(t) ** 2
    thd = sp.Symbol("thd")
    lag = sp.diff(kinetic.subs(th.diff(t), thd), thd).subs(thd, th.diff(t)).diff(t) - kinetic.diff(th)
    # I th'' - (Lagrange left side) = g (the pseudo-force moment moved to the right-hand side)
    g_expr = inert * th.diff(t, 2) - lag
    rng = np.random.default_rng(7)
    for _ in range(5):
        vals = dict(zip(("X2", "a0", "a1", "a2", "th0", "th1", "th2"), rng.standard_normal(7)))
        sub = {X.diff(t, 2): vals["X2"], al.diff(t, 2): vals["a2"], al.diff(t): vals["a1"],
               th.diff(t, 2): vals["th2"], th.diff(t): vals["th1"], al: vals["a0"], th: vals["th0"],
               m: 0.785, l1: 0.55, l2: 0.55, inert: 0.2886}
        g_sym = float(sp.simplify(g_expr.subs(sub)).evalf())
        state = (0.0, 0.0, vals["X2"], vals["a0"], vals["a1"], vals["a2"])
        g_or = okin.pseudo_moment(vals["th0"], state, 0.785, 0.55, 0.55, 0.2886)
        assert abs(g_sym - g_or) < 1e-12 * max(1.0, abs(g_sym))


def test_stationary_driver_reduces_to_plain_torsional_plate():
    """A0 = 0, beta = 0: the passive plate is a torsional plate hanging from a fixed hinge (g = 0)."""
    w = wl.small_flapping(a0=0.0, beta=0.0)
    sim = oracle_sim(w)
    drv = sim.bodies[0]
    pas = sim.bodies[1]
    plain = ofsi.TorsionalBody((0.0, -w["l1"]), -0.5 * np.pi, pas.n_pts, w["ds"], pas.inertia, pas.damping,
                               pas.stiffness, pas.theta)
    rigid = ofsi.RigidBody(drv.pts.copy())
    ref = ofsi.Sim(w["nx"], w["ny"], w["h"], w["x0"], w["y0"], w["n_levels"], w["re"], w["dt"], w["uinf"],
                   w["sd_box"], [rigid, plain], w["ds"])
    for _ in range(4):
        sim.step()
        ref.step()
    for body in (0, 1):
        assert np.array_equal(oracle_history(sim, body), oracle_history(ref, body))


def test_no_slip_on_driven_and_hinged_plates_after_corrector():
    """P E0 (C s + q_inf) equals the prescribed velocities of the driven plate and hinge velocity +
    (alpha1' + theta') q R on the passive plate (Eq. corrector2 enforces the constraint exactly)."""
    w = wl.small_flapping(dt=0.01)
    sim = oracle_sim(w, tol=1e-12)
    for _ in range(3):
        sim.step()
    lev = sim.levels[0]
    u, v = ogrid.faces_from_s(sim.s[0], lev)
    e0q = sim.sd.e0(u + w["uinf"][0], v + w["uinf"][1])
    idx, wts = sim.last_p
    nb = sim.nb
    ub = np.stack([(wts * e0q[idx]).sum(1), (wts * e0q[idx + sim.sd.n_sd]).sum(1)], axis=1)
    drv, pas = sim.bodies
    assert np.max(np.abs(ub[:drv.n_pts] - drv.ur)) < 1e-10
    th = pas.theta                      # last iterate differs from the converged angle by < tol
    ux, uy = pas.u_known(th)
    rx, ry = pas.r(th)
    vel = np.stack([ux + pas.phi * pas.q() * rx, uy + pas.phi * pas.q() * ry], axis=1)
    assert np.max(np.abs(ub[drv.n_pts:nb] - vel)) < 1e-8


def test_flapping_pair_takes_few_fsi_iterations():
    """Sec. 5.1: at most three FSI iterations per step."""
    w = wl.small_flapping()
    sim = oracle_sim(w)
    for _ in range(6):
        sim.step()
    assert max(r["iters"] for r in sim.history) <= 3
