"""Oracle: a deformable body (Sec. 2.1, Eq. beam; App. A) as a geometrically nonlinear beam, FP64 numpy.

Test infrastructure only (see ``oracle/__init__.py``).

The paper discretises Eq. beam with the finite elements of its reference work (not available here).  This
module uses a textbook choice in their place (reading R18): the two-dimensional corotational
Euler-Bernoulli beam element (Crisfield, Non-linear Finite Element Analysis of Solids and Structures,
vol. 1, ch. 7), written from its derivation:

  nodes i = 0..N at spacing ds along the undeformed flag (angle alpha0 from the clamp at node 0), degrees
  of freedom per free node (x_i, y_i, theta_i): position and rotation from the undeformed state.
  Element a-b: chord length L, chord angle beta, rigid rotation psi = beta - beta0, local rotations
  tb_a = theta_a - psi, tb_b = theta_b - psi, axial stretch u = L - L0;
  N = EA u / L0,  (M_a, M_b) = (EI / L0) [[4, 2], [2, 4]] (tb_a, tb_b),
  internal forces  f = N r + M_a e_a + M_b e_b - (M_a + M_b) z / L,
  tangent          K = B^T D B + (N / L) z z^T + ((M_a + M_b) / L^2) (r z^T + z r^T),
  with r = (-c, -s, 0, c, s, 0), z = (s, -c, 0, -s, c, 0), c, s = cos, sin beta, and B the rows r,
  e_a - z/L, e_b - z/L.
  Mass: lumped, mu ds on the translations of every free node (mu ds / 2 at the free end), rotary inertia
  (translational mass) ds^2 / 12.
  Fluid load: body point i is node i; the surface stress f_i (force per unit length by the fluid on the
  body) loads node i's translations with ds f_i (the torsional body's ds-weighted moment of App. A, made
  per point).  Node 0 is clamped; its stress goes to the support.

Time discretisation (Eq. beam4 and the line after it, trapezoidal Newmark):
  (4/dt^2) M chi_{n+1} + R(chi_{n+1}) - ds T^T f = r^zeta_n = M ((4/dt^2) chi_n + (4/dt) zeta_n + zetadot_n)
  (2/dt) chi_{n+1} - zeta_{n+1} = r^chi_n = (2/dt) chi_n + zeta_n
where T picks the translations of the free nodes out of chi (body point i -> node i).  The FSI iteration
(Eqs. stress2, dchi2) linearises R at the iterate chi^(k): J_d = (4/dt^2) M + K(chi^(k)).
"""

import numpy as np


class Beam:
    """Clamped flag of ``n_el`` corotational elements (``n_el + 1`` body points) at spacing ``ds``."""

    kind = "deformable"

    def __init__(self, clamp, alpha0, n_el, ds, mu, ei, ea, tip_angle=0.0):
        self.clamp = np.asarray(clamp, dtype=np.float64)
        self.alpha0 = float(alpha0)
        self.n_el = int(n_el)
        self.n_pts = self.n_el + 1
        self.ds = float(ds)
        self.mu, self.ei, self.ea = float(mu), float(ei), float(ea)
        self.ndof = 3 * self.n_el
        # undeformed node positions
        j = np.arange(self.n_pts, dtype=np.float64) * self.ds
        ca, sa = np.cos(self.alpha0), np.sin(self.alpha0)
        self.x0 = np.stack([self.clamp[0] + j * ca, self.clamp[1] + j * sa], axis=1)
        self.chi = self.initial_shape(tip_angle)
        self.zeta = np.zeros(self.ndof)
        m = self.mass()
        r0, _ = self.internal(self.chi)
        self.zetadot = -r0 / m          # reading R11 for the beam: f_0 = 0, g = 0

    # -- configuration --------------------------------------------------------------------

    def initial_shape(self, tip_angle):
        """Inextensible deflected shape with slope angle phi(s) = tip_angle (2 s - s^2) / L^2 (zero at the
        clamp, tip_angle at the tip, the slope of the small-deflection tip-load shape); node rotations
        phi(s_i), element chords at the mid-element slope, so no element is stretched."""
        length = self.n_el * self.ds
        s = np.arange(self.n_pts, dtype=np.float64) * self.ds
        phi = tip_angle * (2.0 * s / length - (s / length) ** 2)
        smid = s[:-1] + 0.5 * self.ds
        pmid = tip_angle * (2.0 * smid / length - (smid / length) ** 2)
        chi = np.zeros(self.ndof)
        x, y = self.clamp.copy()
        for e in range(self.n_el):
            a = self.alpha0 + pmid[e]
            x, y = x + self.ds * np.cos(a), y + self.ds * np.sin(a)
            chi[3 * e:3 * e + 3] = (x, y, phi[e + 1])
        return chi

    def nodes(self, chi):
        """(n_pts, 3) array of (x, y, theta) of every node, the clamp included."""
        out = np.zeros((self.n_pts, 3))
        out[0, :2] = self.clamp
        out[1:] = chi.reshape(self.n_el, 3)
        return out

    def points(self, chi=None):
        return self.nodes(self.chi if chi is None else chi)[:, :2]

    # -- element and assembly ---------------------------------------------------------------

    def element(self, pa, pb):
        """Internal force (6) and tangent stiffness (6 x 6) of one element from its end nodes (x, y, theta)."""
        l0, beta0 = self.ds, self.alpha0
        dx, dy = pb[0] - pa[0], pb[1] - pa[1]
        length = np.hypot(dx, dy)
        c, s = dx / length, dy / length
        # rigid rotation of the chord, measured from the undeformed direction (no branch cut for |psi| < pi)
        psi = np.arctan2(-dx * np.sin(beta0) + dy * np.cos(beta0), dx * np.cos(beta0) + dy * np.sin(beta0))
        tba, tbb = pa[2] - psi, pb[2] - psi
        u = (length * length - l0 * l0) / (length + l0)
        n = self.ea * u / l0
        ma = self.ei / l0 * (4.0 * tba + 2.0 * tbb)
        mb = self.ei / l0 * (2.0 * tba + 4.0 * tbb)
        r = np.array([-c, -s, 0.0, c, s, 0.0])
        z = np.array([s, -c, 0.0, -s, c, 0.0])
        ea_ = np.array([0.0, 0.0, 1.0, 0.0, 0.0, 0.0])
        eb_ = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
        b = np.stack([r, ea_ - z / length, eb_ - z / length])
        d = np.array([[self.ea / l0, 0.0, 0.0],
                      [0.0, 4.0 * self.ei / l0, 2.0 * self.ei / l0],
                      [0.0, 2.0 * self.ei / l0, 4.0 * self.ei / l0]])
        f = b.T @ np.array([n, ma, mb])
        k = b.T @ d @ b + (n / length) * np.outer(z, z) + ((ma + mb) / length ** 2) * (np.outer(r, z) + np.outer(z, r))
        return f, k

    def internal(self, chi):
        """Assembled internal force R(chi) and tangent K(chi) over the free degrees of freedom."""
        nd = self.nodes(chi)
        r = np.zeros(self.ndof)
        k = np.zeros((self.ndof, self.ndof))
        for e in range(self.n_el):
            fe, ke = self.element(nd[e], nd[e + 1])
            dofs = [3 * (e - 1) + q for q in range(3)] + [3 * e + q for q in range(3)]  # node e, node e+1
            for a_, ga in enumerate(dofs):
                if ga < 0:
                    continue
                r[ga] += fe[a_]
                for b_, gb in enumerate(dofs):
                    if gb >= 0:
                        k[ga, gb] += ke[a_, b_]
        return r, k

    def mass(self):
        """Lumped mass (diagonal) over the free degrees of freedom."""
        m = np.empty(self.ndof)
        for i in range(self.n_el):
            mt = self.mu * self.ds * (0.5 if i == self.n_el - 1 else 1.0)
            m[3 * i:3 * i + 3] = (mt, mt, mt * self.ds ** 2 / 12.0)
        return m

    def t_matrix(self, nb_total, offset):
        """T: (n_el*3) x (2 nb_total) map from the stress vector to the nodal loads / velocities, so that
        (T^T)... is used as T @ zeta (point velocities) and T.T @ f (nodal loads before ds)."""
        t = np.zeros((2 * nb_total, self.ndof))
        for i in range(1, self.n_pts):
            p = offset + i
            t[p, 3 * (i - 1)] = 1.0
            t[nb_total + p, 3 * (i - 1) + 1] = 1.0
        return t

    # -- time stepping -------------------------------------------------------------------------

    def jac(self, dt, chi):
        _, k = self.internal(chi)
        return np.diag(4.0 / dt ** 2 * self.mass()) + k

    def rhs_terms(self, dt):
        """r^zeta_n and r^chi_n (Newmark, App. A; g = 0)."""
        m = self.mass()
        r_zeta = m * (4.0 / dt ** 2 * self.chi + 4.0 / dt * self.zeta + self.zetadot)
        r_chi = 2.0 / dt * self.chi + self.zeta
        return r_zeta, r_chi

    def advance(self, chi_new, r_chi, dt):
        zeta_new = 2.0 / dt * chi_new - r_chi
        self.zetadot = 4.0 / dt ** 2 * (chi_new - self.chi) - 4.0 / dt * self.zeta - self.zetadot
        self.chi, self.zeta = chi_new, zeta_new

    # -- outputs -------------------------------------------------------------------------------

    def tip_deflection(self, chi=None, zeta=None):
        """Transverse displacement of the tip from the undeformed line and its rate."""
        chi = self.chi if chi is None else chi
        zeta = self.zeta if zeta is None else zeta
        nrm = np.array([-np.sin(self.alpha0), np.cos(self.alpha0)])
        tip = chi[-3:-1]
        return float((tip - self.x0[-1]) @ nrm), float(zeta[-3:-1] @ nrm)

    def energy(self, chi=None, zeta=None):
        """Kinetic + strain energy (strain energy of each element from its local deformations)."""
        chi = self.chi if chi is None else chi
        zeta = self.zeta if zeta is None else zeta
        kin = 0.5 * float(np.sum(self.mass() * zeta * zeta))
        nd = self.nodes(chi)
        pot = 0.0
        for e in range(self.n_el):
            pa, pb = nd[e], nd[e + 1]
            dx, dy = pb[0] - pa[0], pb[1] - pa[1]
            length = np.hypot(dx, dy)
            b0 = self.alpha0
            psi = np.arctan2(-dx * np.sin(b0) + dy * np.cos(b0), dx * np.cos(b0) + dy * np.sin(b0))
            tba, tbb = pa[2] - psi, pb[2] - psi
            u = (length * length - self.ds ** 2) / (length + self.ds)
            pot += 0.5 * self.ea * u * u / self.ds
            pot += 0.5 * self.ei / self.ds * (4 * tba * tba + 4 * tba * tbb + 4 * tbb * tbb)
        return kin + pot
