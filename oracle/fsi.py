"""Oracle: bodies, the FSI iteration and the time step (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

One step n -> n+1 follows Algorithm 2 with Eqs. predictor2, stress2, dtheta2
and corrector2; the structural right-hand sides follow App. A:

  O1  fine->coarse vorticity injection (multidomain, reading R5)
  O2  advection term and right-hand side on every level (App. A, AB2 + CN)
  O3  predictor, coarse to fine: ``s* = (C^T A C)^{-1} r`` (Eq. predictor2)
  O4  FSI iteration on the finest level (Eqs. stress2, dtheta2) with
      ``P B0 P^T`` in place of ``E C (C^T A C)^{-1} C^T E^T`` (Eq. operatorapprox);
      with a drop tolerance the filtered ``B0'`` of Eq. filtereq (then K is not symmetric)
  O5  corrector ``s = s* - (C^T A C)^{-1} C^T E0^T P^T f`` (Eq. corrector2) on the
      finest level with homogeneous boundary values (reading R6)
  O6  Newmark update of the structure and the force outputs

Bodies: rigid (prescribed velocity), torsional plate (App. A, reading R3) and the
deformable flag of ``oracle/beam.py`` (App. A with J_d, S_d, reading R18).  The
iteration stops on max abs of the structural update (reading R14).

Scaling of the coupling (reading R2): the fluid forcing on faces is
``-(ds/h^2) E^T f``; ``f`` is the force per unit length exerted by the fluid on
the body, so the total force on a body is ``ds * sum_j f_j`` and
``c_d = 2 F_x``, ``c_l = 2 F_y`` (reading R4, rho = U = c = 1).
Torsional coupling operator (reading R3): ``S = Q R`` with ``Q_j = j ds`` and
``R_j = (-sin, cos)(theta0 + theta)``.
"""

import numpy as np

from . import grid, ib


class TorsionalBody:
    """Flat plate of ``n_pts`` points at spacing ``ds`` hinged at ``hinge`` (App. A)."""

    kind = "torsional"

    def __init__(self, hinge, theta0, n_pts, ds, inertia, damping, stiffness, theta, phi=0.0):
        self.hinge = np.asarray(hinge, dtype=np.float64)
        self.theta0 = float(theta0)
        self.n_pts = int(n_pts)
        self.ds = float(ds)
        self.inertia, self.damping, self.stiffness = float(inertia), float(damping), float(stiffness)
        self.theta = float(theta)
        self.phi = float(phi)
        # reading R11: f_0 = 0, g_t = 0, so the initial acceleration balances the spring and damper
        self.phidot = (-self.stiffness * self.theta - self.damping * self.phi) / self.inertia

    def g(self, theta):
        """Moment of body forces (g_t of Eq. newtons): zero for a plate on a fixed hinge (reading R17)."""
        return 0.0

    def u_known(self, theta):
        """Point velocities apart from theta' S: zero on a fixed hinge."""
        return 0.0, 0.0

    def points(self, theta):
        j = np.arange(self.n_pts, dtype=np.float64) * self.ds
        a = self.theta0 + theta
        return np.stack([self.hinge[0] + j * np.cos(a), self.hinge[1] + j * np.sin(a)], axis=1)

    def q(self):
        """Moment arms ``Q = [0, 1, ..., n] ds`` (App. A)."""
        return np.arange(self.n_pts, dtype=np.float64) * self.ds

    def r(self, theta):
        """Normal-projection entries ``(-sin, cos)(theta0 + theta)`` (App. A)."""
        a = self.theta0 + theta
        return -np.sin(a), np.cos(a)

    def jac(self, dt):
        """``J = 4 I/dt^2 + 2 c/dt + k`` (App. A)."""
        return 4.0 * self.inertia / dt ** 2 + 2.0 * self.damping / dt + self.stiffness

    def rhs_terms(self, dt):
        """``r^{phidot}_n`` and ``r^{theta}_n`` of App. A (``g_t = 0``, reading R17)."""
        r_phi = (self.inertia * (4.0 * self.theta / dt ** 2 + 4.0 * self.phi / dt + self.phidot)
                 + self.damping * (2.0 * self.theta / dt + self.phi))
        r_theta = self.phi + 2.0 / dt * self.theta
        return r_phi, r_theta

    def advance(self, theta_new, r_theta, dt):
        """Newmark (trapezoidal) update to step n+1 given the converged angle (reading R11)."""
        phi_new = 2.0 / dt * theta_new - r_theta
        self.phidot = 4.0 / dt ** 2 * (theta_new - self.theta) - 4.0 / dt * self.phi - self.phidot
        self.theta, self.phi = theta_new, phi_new


class RigidBody:
    """Points with a prescribed velocity ``ur`` (zero for a stationary body)."""

    kind = "rigid"

    def __init__(self, pts, ur=None, appended=False):
        self.pts = np.asarray(pts, dtype=np.float64)
        self.n_pts = len(self.pts)
        self.ur = np.zeros_like(self.pts) if ur is None else np.asarray(ur, dtype=np.float64)
        self.ds = None
        # appended: the points join Omega_0 and are interpolated with E itself (Sec. 3.1.1)
        self.appended = bool(appended)

    def points(self, theta=None):
        return self.pts


class NotConverged(RuntimeError):
    pass


class Sim:
    """A full run: nested levels, one sub-domain box, bodies, FP64 state."""

    def __init__(self, nx, ny, h, x0, y0, n_levels, re, dt, uinf, sd_box, bodies, ds,
                 tol=1e-7, max_iters=50, drop_tol=0.0, coupling="subdomain"):
        self.levels = grid.make_levels(nx, ny, h, x0, y0, n_levels)
        self.re, self.dt = float(re), float(dt)
        self.uinf = np.asarray(uinf, dtype=np.float64)
        self.ds = float(ds)
        self.bodies = list(bodies)
        self.tol, self.max_iters = float(tol), int(max_iters)
        self.drop_tol = float(drop_tol)      # Eq. filtereq: B0' in place of B0 in the small system
        # "subdomain": E ~ P E0 (Eq. operatorapprox); "true": E at the body points, the small matrix
        # E C (C^T A C)^-1 C^T E^T built column by column (the comparator of Sec. 5.1)
        self.coupling = coupling
        self.last_pts = None
        # exact points of stationary bodies appended to Omega_0 (Sec. 3.1.1), in body order
        app = [b.pts for b in self.bodies if getattr(b, "appended", False)]
        extra = np.concatenate(app) if app else None
        if sd_box is None:
            self.sd = None
        elif np.ndim(sd_box) == 2:           # a union of boxes (reading R16)
            self.sd = ib.Subdomain.from_boxes(self.levels[0], sd_box, extra=extra)
        else:
            self.sd = ib.Subdomain.from_box(self.levels[0], *sd_box, extra=extra)
        self.appended = np.full(sum(b.n_pts for b in self.bodies), -1, dtype=np.int64)
        o = e = 0
        for b in self.bodies:
            if getattr(b, "appended", False):
                self.appended[o:o + b.n_pts] = e + np.arange(b.n_pts)
                e += b.n_pts
            o += b.n_pts
        self.w = [np.zeros(l.shape) for l in self.levels]
        self.s = [np.zeros(l.shape) for l in self.levels]
        self.nprev = [None] * len(self.levels)
        self.nb = sum(b.n_pts for b in self.bodies)
        self.f = np.zeros(2 * self.nb)
        self._b0 = {}
        self.history = []
        self.last_p = None
        self.last_svec = {}
        self.t = 0.0                          # time of the current state (bodies with kinematics)

    # -- B0 columns, computed on first use and cached (Eq. action) ---------------------

    def b0_cols(self, cols):
        out = np.empty((2 * self.sd.n_sd, len(cols)))
        for k, c in enumerate(cols):
            c = int(c)
            if c not in self._b0:
                self._b0[c] = ib.b0_column(self.sd, c, self.re, self.dt, self.drop_tol)
            out[:, k] = self._b0[c]
        return out

    # -- O1-O3 -------------------------------------------------------------------------

    def predictor(self):
        L, G, dt, re = self.levels, len(self.levels), self.dt, self.re
        for g in range(G - 1):
            grid.inject_fine_to_coarse(self.w[g], L[g], self.w[g + 1], L[g + 1])
        rhs = []
        for g in range(G):
            n_now = grid.nonlinear(self.s[g], self.w[g], L[g], self.uinf)
            n_old = n_now if self.nprev[g] is None else self.nprev[g]
            r = (self.w[g][1:-1, 1:-1] / dt + grid.laplacian(self.w[g], L[g]) / (2.0 * re)
                 - 1.5 * n_now + 0.5 * n_old)
            self.nprev[g] = n_now
            rhs.append(r)
        for g in range(G - 1, -1, -1):
            if g < G - 1:
                grid.set_ring_from_coarse(self.w[g], L[g], self.w[g + 1], L[g + 1])
                grid.set_ring_from_coarse(self.s[g], L[g], self.s[g + 1], L[g + 1])
            w_int = grid.solve_aw(rhs[g], self.w[g], L[g], re, dt)
            self.w[g][1:-1, 1:-1] = w_int
            self.s[g][1:-1, 1:-1] = grid.solve_lap(w_int, self.s[g], L[g])

    # -- O4: FSI iteration (Eqs. stress2, dtheta2) ---------------------------------------

    def _body_offsets(self):
        off, o = [], 0
        for b in self.bodies:
            off.append(o)
            o += b.n_pts
        return off

    def fsi(self):
        lev, sd, dt, ds, nb = self.levels[0], self.sd, self.dt, self.ds, self.nb
        for b in self.bodies:                       # prescribed kinematics at t_{n+1}
            if hasattr(b, "at_time"):
                b.at_time(self.t + dt)
        u, v = grid.faces_from_s(self.s[0], lev)
        e0q = sd.e0(u + self.uinf[0], v + self.uinf[1]) if self.coupling != "true" else None  # E0 (C s* + q_inf)
        offs = self._body_offsets()
        moving = [(b, o) for b, o in zip(self.bodies, offs) if b.kind != "rigid"]
        # iterate state: theta (torsional) or chi (deformable), and its rate phi or zeta
        state_k = {id(b): (b.theta if b.kind == "torsional" else b.chi.copy()) for b, _ in moving}
        rate_k = {id(b): (b.phi if b.kind == "torsional" else b.zeta.copy()) for b, _ in moving}
        for it in range(self.max_iters):
            pts = np.concatenate([b.points(state_k.get(id(b))) for b in self.bodies])
            if self.coupling == "true":
                kmat = (ds / lev.h ** 2) * np.stack(
                    [ib.ke_column(lev, pts, m, self.re, self.dt) for m in range(2 * nb)], axis=1)
                rhs = ib.e_points(lev, pts, u + self.uinf[0], v + self.uinf[1])   # E (C s* + q_inf)
                idx = wts = None
            else:
                idx, wts = sd.p_rows(pts, self.appended)
                cols = np.unique(np.concatenate([idx.ravel(), idx.ravel() + sd.n_sd]))
                pos = {c: k for k, c in enumerate(cols)}
                pd = np.zeros((2 * nb, len(cols)))
                for p in range(nb):
                    for k in range(4):
                        pd[p, pos[idx[p, k]]] += wts[p, k]
                        pd[nb + p, pos[idx[p, k] + sd.n_sd]] += wts[p, k]
                kmat = (ds / lev.h ** 2) * pd @ self.b0_cols(cols)[cols, :] @ pd.T
                rhs = pd @ e0q[cols]                                   # P E0 (C s* + q_inf)
            svec, dstate = {}, {}
            for b, o in zip(self.bodies, offs):
                if b.kind == "rigid":
                    rhs[o:o + b.n_pts] -= b.ur[:, 0]
                    rhs[nb + o:nb + o + b.n_pts] -= b.ur[:, 1]
                    continue
                if b.kind == "deformable":
                    # App. A with J_d = 4 M/dt^2 + K(chi^(k)) and the load map T (reading R18):
                    # K += (2 ds/dt) T J_d^-1 T^T,  r^c(k) = T ((2/dt)(chi^(k) + J_d^-1 r^zeta(k)) - r^chi)
                    chi = state_k[id(b)]
                    rint, ktan = b.internal(chi)
                    m = b.mass()
                    jd = np.diag(4.0 / dt ** 2 * m) + ktan
                    rz = self._r_phi[id(b)] - 4.0 / dt ** 2 * m * chi - rint      # r^zeta(k)
                    tm = b.t_matrix(nb, o)
                    kmat += (2.0 * ds / dt) * tm @ np.linalg.solve(jd, tm.T)
                    rhs -= tm @ (2.0 / dt * (chi + np.linalg.solve(jd, rz)) - self._r_theta[id(b)])
                    dstate[id(b)] = (jd, rz, tm)
                    continue
                th, ph = state_k[id(b)], rate_k[id(b)]
                rx, ry = b.r(th)
                sv = np.zeros(2 * nb)
                sv[o:o + b.n_pts] = b.q() * rx
                sv[nb + o:nb + o + b.n_pts] = b.q() * ry
                svec[id(b)] = sv
                ukx, uky = b.u_known(th)                                 # moving hinge (reading R20)
                rhs[o:o + b.n_pts] -= ukx
                rhs[nb + o:nb + o + b.n_pts] -= uky
                jac = b.jac(dt)
                r_phi = self._r_phi[id(b)] + b.g(th) - jac * th          # r^{phidot}(k), g at the iterate
                r_theta = self._r_theta[id(b)] - 2.0 / dt * th + ph      # r^{theta}(k)
                kmat += (2.0 * ds / dt) / jac * np.outer(sv, sv)
                rhs -= sv * ph                                           # r^c(k) = R^T Q^T phi^(k)
                rhs += sv * (r_theta - 2.0 / dt * r_phi / jac)
            f = np.linalg.solve(kmat, rhs)
            dmax = 0.0
            for b, _ in moving:
                if b.kind == "deformable":
                    jd, rz, tm = dstate[id(b)]
                    dchi = np.linalg.solve(jd, rz + ds * tm.T @ f)                  # Eq. dchi2
                    state_k[id(b)] = state_k[id(b)] + dchi
                    rate_k[id(b)] = 2.0 / dt * state_k[id(b)] - self._r_theta[id(b)]
                    dmax = max(dmax, float(np.max(np.abs(dchi))))
                    continue
                th = state_k[id(b)]
                jac = b.jac(dt)
                dth = (self._r_phi[id(b)] + b.g(th) - jac * th + ds * svec[id(b)] @ f) / jac   # Eq. dtheta2
                state_k[id(b)] = th + dth
                rate_k[id(b)] = 2.0 / dt * state_k[id(b)] - self._r_theta[id(b)]
                dmax = max(dmax, abs(dth))
            self.last_p = (idx, wts)
            self.last_pts = pts
            self.last_svec = svec
            self.last_dmax = dmax
            if dmax <= self.tol:
                return f, state_k, rate_k, it + 1
        raise NotConverged("FSI iteration did not converge")

    # -- O5: corrector (Eq. corrector2) --------------------------------------------------

    def corrector(self, f):
        lev, sd, nb = self.levels[0], self.sd, self.nb
        if self.coupling == "true":
            u, v = ib.et_points(lev, self.last_pts, f)          # E^T f at the last iterate's points
        else:
            idx, wts = self.last_p
            g = np.zeros(2 * sd.n_sd)
            for p in range(nb):                                  # P^T f
                for k in range(4):
                    g[idx[p, k]] += wts[p, k] * f[p]
                    g[idx[p, k] + sd.n_sd] += wts[p, k] * f[nb + p]
            u, v = sd.e0t(g)
        src = (self.ds / lev.h ** 2) * grid.curl_faces(u, v, lev)
        zero = np.zeros(lev.shape)
        dw = grid.solve_aw(src, zero, lev, self.re, self.dt)
        ds_ = grid.solve_lap(dw, zero, lev)
        self.w[0][1:-1, 1:-1] -= dw
        self.s[0][1:-1, 1:-1] -= ds_

    # -- one full step (Algorithm 2) -----------------------------------------------------

    def step(self):
        dt = self.dt
        self._r_phi, self._r_theta = {}, {}
        for b in self.bodies:
            if b.kind != "rigid":
                # torsional: r^{phidot}_n, r^theta_n; deformable: r^zeta_n, r^chi_n (App. A)
                self._r_phi[id(b)], self._r_theta[id(b)] = b.rhs_terms(dt)
        self.predictor()
        n_it = 0
        if self.bodies:
            f, theta_k, phi_k, n_it = self.fsi()
            self.corrector(f)
            self.f = f
            for b in self.bodies:
                if b.kind != "rigid":
                    b.advance(theta_k[id(b)], self._r_theta[id(b)], dt)
        rec = {"iters": n_it, "bodies": []}
        offs = self._body_offsets()
        for b, o in zip(self.bodies, offs):
            fx = self.ds * np.sum(self.f[o:o + b.n_pts])
            fy = self.ds * np.sum(self.f[self.nb + o:self.nb + o + b.n_pts])
            mom = 0.0
            if b.kind == "torsional" and self.last_svec:
                mom = self.ds * float(self.last_svec[id(b)] @ self.f)       # ds S f, S at the last iterate
            if b.kind == "deformable":
                tip, tip_rate = b.tip_deflection()
                rec["bodies"].append({"fx": fx, "fy": fy, "moment": 0.0, "theta": tip, "phi": tip_rate})
                continue
            rec["bodies"].append({"fx": fx, "fy": fy, "moment": mom,
                                  "theta": getattr(b, "theta", 0.0), "phi": getattr(b, "phi", 0.0)})
        self.history.append(rec)
        self.t += dt
        return rec
