"""Oracle: prescribed flapping kinematics of the driven plate and the hinged passive plate (Sec. 5.1,
Eq. newtonseldg).  FP64, numpy/scipy.  Test infrastructure only (see ``oracle/__init__.py``).

Driven plate (a rigid body with prescribed motion): its reference point (the pitch axis / centre of the
ellipse it stands in for) is at ``(xc + X1(t), yc)``; the plate lies along ``e(alpha1) = (sin, -cos)(alpha1)``
(straight down at alpha1 = 0) from ``s_lo`` to ``s_hi`` (the hinge end).  With tau = f t:

  X1(t)     = (A0/2) G_t(tau) / max G_t * C(tau)        Y1 = 0
  alpha1(t) = -beta G_r(tau) / max G_r
  G_t(tau)  = int_0^tau tanh(sigma_t cos(2 pi u)) du    (zero mean over a period, so periodic)
  G_r(tau)  = tanh(sigma_r cos(2 pi tau))
  C(tau)    = (tanh(8 tau - 2) + tanh 2) / (1 + tanh 2)  (start-up conditioner)

Passive plate: a torsional plate hinged at ``hinge(t) = ref(t) + L1 e(alpha1)``, lying along
``e(alpha1 + theta)``; its rest direction is therefore theta0(t) = alpha1(t) - pi/2 in the convention of
the plain torsional plate (direction (cos, sin)(theta0 + theta)).  Its equation about the hinge
(Eq. newtonseldg, reading R20) is

  I theta'' + c theta' + k theta = M_f + g(theta, t),
  g = -m L2 cos(alpha1 + theta) X1'' - (I + m L1 L2 cos theta) alpha1'' - m L1 L2 sin theta alpha1'^2

with I the moment of inertia about the hinge (the paper's I_cg + m L2^2 in the bracket) and m, L2 the
passive plate's mass and the distance of its centre of mass from the hinge.  Points of the passive plate
move with the hinge velocity plus the rotation (alpha1' + theta') about the hinge.
"""

import numpy as np
from scipy import integrate

from .fsi import TorsionalBody


class FlappingKinematics:
    """X1, alpha1 and their first two time derivatives (Sec. 5.1)."""

    def __init__(self, a0, beta, sigma_t, sigma_r, freq=1.0):
        self.a0, self.beta = float(a0), float(beta)
        self.sigma_t, self.sigma_r, self.freq = float(sigma_t), float(sigma_r), float(freq)
        self.gt_max = self.g_t(0.25)            # G_t rises while cos > 0, i.e. up to tau = 1/4
        self.gr_max = np.tanh(self.sigma_r)     # G_r is largest at tau = 0

    def g_t(self, tau):
        """G_t by adaptive quadrature over the fractional part of tau (a period integrates to zero)."""
        frac = float(tau) - np.floor(float(tau))
        val, _ = integrate.quad(lambda u: np.tanh(self.sigma_t * np.cos(2.0 * np.pi * u)), 0.0, frac,
                                epsabs=1e-14, epsrel=1e-13, limit=200)
        return val

    def conditioner(self, tau):
        """C, C', C'' with respect to tau."""
        th2 = np.tanh(2.0)
        z = 8.0 * tau - 2.0
        tz = np.tanh(z)
        sech2 = 1.0 - tz * tz
        c0 = (tz + th2) / (1.0 + th2)
        c1 = 8.0 * sech2 / (1.0 + th2)
        c2 = -128.0 * sech2 * tz / (1.0 + th2)
        return c0, c1, c2

    def state(self, t):
        """(X1, X1', X1'', alpha1, alpha1', alpha1'') at time t (derivatives in t)."""
        f = self.freq
        tau = f * float(t)
        w = 2.0 * np.pi
        st, ct = np.sin(w * tau), np.cos(w * tau)
        # G_t and its tau-derivatives
        g0 = self.g_t(tau)
        ut = self.sigma_t * ct
        tt = np.tanh(ut)
        g1 = tt
        g2 = -w * self.sigma_t * st * (1.0 - tt * tt)
        c0, c1, c2 = self.conditioner(tau)
        ax = 0.5 * self.a0 / self.gt_max
        x = ax * g0 * c0
        xd = f * ax * (g1 * c0 + g0 * c1)
        xdd = f * f * ax * (g2 * c0 + 2.0 * g1 * c1 + g0 * c2)
        # G_r and its tau-derivatives
        ur = self.sigma_r * ct
        tr = np.tanh(ur)
        s2 = 1.0 - tr * tr
        du = -w * self.sigma_r * st
        r0 = tr
        r1 = s2 * du
        r2 = -w * w * self.sigma_r * ct * s2 - 2.0 * s2 * tr * du * du
        ar = -self.beta / self.gr_max
        return x, xd, xdd, ar * r0, f * ar * r1, f * f * ar * r2


def e_dir(a):
    """Unit vector along a plate at angle a: (sin a, -cos a) (straight down at a = 0)."""
    return np.array([np.sin(a), -np.cos(a)])


def e_rot(a):
    """d e_dir / da = (cos a, sin a): the direction of positive rotation."""
    return np.array([np.cos(a), np.sin(a)])


class DrivenPlate:
    """Rigid plate with the prescribed heave and pitch (a rigid body whose points and velocities change
    with time).  Points at s_j = s_lo + j ds, j = 0 .. n_pts - 1, along e(alpha1) from the reference point."""

    kind = "rigid"

    def __init__(self, ref, s_lo, n_pts, ds, kin):
        self.ref = np.asarray(ref, dtype=np.float64)
        self.s_lo = float(s_lo)
        self.n_pts = int(n_pts)
        self.ds = float(ds)
        self.kin = kin
        self.at_time(0.0)

    def s(self):
        return self.s_lo + np.arange(self.n_pts, dtype=np.float64) * self.ds

    def at_time(self, t):
        """Set the points and their velocities to the kinematics at time t."""
        self.state = self.kin.state(t)
        x, xd, _, a, ad, _ = self.state
        s = self.s()
        e, er = e_dir(a), e_rot(a)
        self.pts = np.stack([self.ref[0] + x + s * e[0], self.ref[1] + s * e[1]], axis=1)
        self.ur = np.stack([xd + s * ad * er[0], s * ad * er[1]], axis=1)

    def points(self, theta=None):
        return self.pts


def pseudo_moment(theta, kin_state, mass, l1, l2, inertia):
    """g of Eq. newtonseldg: moments of the pseudo-forces on the passive plate about the moving hinge."""
    _, _, xdd, a, ad, add = kin_state
    return (-mass * l2 * np.cos(a + theta) * xdd - (inertia + mass * l1 * l2 * np.cos(theta)) * add
            - mass * l1 * l2 * np.sin(theta) * ad * ad)


class HingedPlate(TorsionalBody):
    """Passive plate hinged at distance l1 along the driven plate from its reference point (Eq. newtonseldg).
    theta is the deflection from the driven plate's direction; mass and l2 (centre of mass from the hinge)
    enter the pseudo-force moment g, inertia is about the hinge."""

    def __init__(self, driver, l1, n_pts, ds, inertia, damping, stiffness, mass, l2, theta, phi=0.0):
        self.driver = driver
        self.l1, self.mass, self.l2 = float(l1), float(mass), float(l2)
        self.at_time(0.0)
        super().__init__(self.hinge, self.theta0, n_pts, ds, inertia, damping, stiffness, theta, phi)
        # reading R11 with the pseudo-forces: f_0 = 0, so I phi'(0) = -k theta - c phi + g(theta, 0)
        self.phidot += self.g(self.theta) / self.inertia

    def at_time(self, t):
        """Hinge position and velocity, rest direction theta0 = alpha1 - pi/2 and the kinematics at t."""
        self.kin_state = self.driver.kin.state(t)
        x, xd, _, a, ad, _ = self.kin_state
        e, er = e_dir(a), e_rot(a)
        self.hinge = np.array([self.driver.ref[0] + x + self.l1 * e[0], self.driver.ref[1] + self.l1 * e[1]])
        self.v_hinge = np.array([xd + self.l1 * ad * er[0], self.l1 * ad * er[1]])
        self.theta0 = a - 0.5 * np.pi
        self.alpha_dot = ad

    def g(self, theta):
        return pseudo_moment(theta, self.kin_state, self.mass, self.l1, self.l2, self.inertia)

    def u_known(self, theta):
        """Velocity of the points apart from theta' S: hinge velocity + alpha1' q R(theta)."""
        rx, ry = self.r(theta)
        q = self.q()
        return self.v_hinge[0] + self.alpha_dot * q * rx, self.v_hinge[1] + self.alpha_dot * q * ry
