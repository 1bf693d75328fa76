"""Oracle: staggered-grid streamfunction/vorticity fluid operators (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

Discretisation (Sec. 2.2 and App. A of the paper; the operators themselves are
deferred there to Taira & Colonius, so the concrete scaling below is this
project's reading):

* A level has ``nx x ny`` cells of spacing ``h`` with lower-left corner
  ``(x0, y0)``.  Streamfunction ``s`` and vorticity ``w`` live on the vertices
  ``(x0 + i h, y0 + j h)``, ``i = 0..nx``, ``j = 0..ny``; arrays are indexed
  ``[j, i]`` and include the boundary ring.
* Velocity fluxes on faces, ``q = C s``:
  ``u[j, i] = (s[j+1, i] - s[j, i]) / h``   at ``(x_i, y_{j+1/2})``,
  ``v[j, i] = -(s[j, i+1] - s[j, i]) / h``  at ``(x_{i+1/2}, y_j)``.
* The discrete curl is ``C^T``; ``C^T C = -lap_h`` (5-point Laplacian).
* Crank-Nicolson viscous operator on vorticity
  ``A_w = 1/dt - lap_h / (2 Re)`` so that ``C^T A C = (C^T C) A_w`` and
  ``(C^T A C)^{-1} = Lap^{-1} A_w^{-1}`` (Sec. 3.2.1: ``A = I + alpha C C^T``).
* Both inverses are diagonal in the 2-D DST-I basis (Sec. 3.2.1,
  ``C^T C = S Lambda S^T``).  The oracle applies the DST as a dense product
  with the sine matrix.

Multidomain (Sec. 5 intro, Colonius & Taira far-field scheme; reading R5):
``G`` levels share ``nx x ny`` and the centre, ``h_g = 2^g h``.  Each step the
coarse vorticity strictly inside a finer level is replaced by injection from the
coincident fine vertex; the coarsest level has zero boundary values; every other
level takes its boundary ``w`` and ``s`` from the next coarser level (injection
at coincident vertices, linear interpolation at midpoints).  Each step the
sweep runs coarse to fine, so a finer level's ring holds the coarser level at
t^{n+1}.  The coupling is pinned by a Lamb-Oseen vortex, an exact
Navier-Stokes solution (``tests/test_oracle_multidomain.py``: error vs the
number of levels, second order in h and in dt, fine accuracy of the coarse
level inside the finer one, rings at the new time); the rest of this file by
``tests/test_oracle_pins.py``.
"""

import numpy as np


class Level:
    """One uniform level: ``nx x ny`` cells, spacing ``h``, corner ``(x0, y0)``."""

    def __init__(self, nx, ny, h, x0, y0):
        self.nx, self.ny, self.h, self.x0, self.y0 = int(nx), int(ny), float(h), float(x0), float(y0)

    @property
    def shape(self):
        return (self.ny + 1, self.nx + 1)

    def xv(self):
        return self.x0 + self.h * np.arange(self.nx + 1)

    def yv(self):
        return self.y0 + self.h * np.arange(self.ny + 1)


def make_levels(nx, ny, h, x0, y0, n_levels):
    """Nested levels sharing the centre of the finest one; level g has spacing 2^g h."""
    cx, cy = x0 + 0.5 * nx * h, y0 + 0.5 * ny * h
    out = []
    for g in range(n_levels):
        hg = h * (2 ** g)
        out.append(Level(nx, ny, hg, cx - 0.5 * nx * hg, cy - 0.5 * ny * hg))
    return out


# ---------------------------------------------------------------------------
# DST-I (Sec. 3.2.1: the eigenvectors of C^T C are discrete sine transforms)
# ---------------------------------------------------------------------------

def dst1_matrix(n):
    """Unnormalised DST-I matrix ``S[j-1, k-1] = sin(pi j k / (n+1))``; ``S S = (n+1)/2 I``."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return np.sin(np.pi * np.outer(k, k) / (n + 1))


def lap_eigs_1d(n, h):
    """Eigenvalues of the 1-D Dirichlet operator ``-(d^2/dx^2)_h`` on ``n`` interior points."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return 4.0 / (h * h) * np.sin(np.pi * k / (2.0 * (n + 1))) ** 2


def dirichlet_diag_solve(rhs, diag):
    """Solve ``D x = rhs`` where ``D`` is diagonal (entries ``diag[l, k]``) in the 2-D DST-I basis.

    ``rhs`` and ``diag`` have shape ``(Ny, Nx)`` (interior vertices, rows = y).
    Forward transform, divide, inverse transform with the ``(2/M)`` normalisation per axis.
    """
    ny_, nx_ = rhs.shape
    sy, sx = dst1_matrix(ny_), dst1_matrix(nx_)
    r_hat = sy @ rhs @ sx
    return (4.0 / ((ny_ + 1) * (nx_ + 1))) * (sy @ (r_hat / diag) @ sx)


def lap_diag(lev):
    """``lambda_kl`` of ``-lap_h`` on the interior of ``lev`` as an ``(Ny, Nx)`` array."""
    lx = lap_eigs_1d(lev.nx - 1, lev.h)
    ly = lap_eigs_1d(lev.ny - 1, lev.h)
    return ly[:, None] + lx[None, :]


def aw_diag(lev, re, dt):
    """Eigenvalues of ``A_w = 1/dt - lap_h/(2 Re)`` (Crank-Nicolson, Sec. 3.2.1)."""
    return 1.0 / dt + lap_diag(lev) / (2.0 * re)


def ring_neighbour_sum(full):
    """For each interior vertex, the sum of its 5-point neighbours that lie on the boundary ring."""
    out = np.zeros((full.shape[0] - 2, full.shape[1] - 2))
    out[:, 0] += full[1:-1, 0]
    out[:, -1] += full[1:-1, -1]
    out[0, :] += full[0, 1:-1]
    out[-1, :] += full[-1, 1:-1]
    return out


def solve_aw(rhs, w_ring_full, lev, re, dt):
    """Interior ``w`` with ``A_w w = rhs`` given boundary values ``w_ring_full`` (full array, ring used)."""
    r = rhs + ring_neighbour_sum(w_ring_full) / (2.0 * re * lev.h ** 2)
    return dirichlet_diag_solve(r, aw_diag(lev, re, dt))


def solve_lap(w_int, s_ring_full, lev):
    """Interior ``s`` with ``-lap_h s = w`` given boundary values ``s_ring_full``."""
    r = w_int + ring_neighbour_sum(s_ring_full) / lev.h ** 2
    return dirichlet_diag_solve(r, lap_diag(lev))


# ---------------------------------------------------------------------------
# C, C^T, Laplacian, nonlinear term
# ---------------------------------------------------------------------------

def faces_from_s(s, lev):
    """``q = C s`` with ``s`` the full vertex array (ring included)."""
    h = lev.h
    u = (s[1:, :] - s[:-1, :]) / h          # (ny, nx+1): u[j, i] at (x_i, y_{j+1/2})
    v = -(s[:, 1:] - s[:, :-1]) / h         # (ny+1, nx): v[j, i] at (x_{i+1/2}, y_j)
    return u, v


def curl_faces(u, v, lev):
    """``C^T q`` at interior vertices: ``dv/dx - du/dy``."""
    h = lev.h
    dvdx = (v[1:-1, 1:] - v[1:-1, :-1]) / h     # v[j, i] - v[j, i-1], j=1..ny-1, i=1..nx-1
    dudy = (u[1:, 1:-1] - u[:-1, 1:-1]) / h     # u[j, i] - u[j-1, i]
    return dvdx - dudy


def laplacian(w, lev):
    """5-point ``lap_h w`` at interior vertices (ring values of ``w`` used)."""
    return (w[1:-1, 2:] + w[1:-1, :-2] + w[2:, 1:-1] + w[:-2, 1:-1] - 4.0 * w[1:-1, 1:-1]) / lev.h ** 2


def nonlinear(s, w, lev, uinf):
    """Advection term ``N = div(u w)`` at interior vertices (reading R7).

    Vertex velocities: ``ubar`` = mean of the u-faces just above and below
    plus ``U_inf,x``; ``vbar`` = mean of the v-faces just left and right plus
    ``U_inf,y``.  Central differences of the fluxes ``ubar w`` and ``vbar w``.
    """
    h = lev.h
    u, v = faces_from_s(s, lev)
    ubar = 0.5 * (u[1:, :] + u[:-1, :]) + uinf[0]        # rows j=1..ny-1, all i
    vbar = 0.5 * (v[:, 1:] + v[:, :-1]) + uinf[1]        # all j, cols i=1..nx-1
    fx = ubar * w[1:-1, :]                               # (ny-1, nx+1)
    fy = vbar * w[:, 1:-1]                               # (ny+1, nx-1)
    return (fx[:, 2:] - fx[:, :-2]) / (2 * h) + (fy[2:, :] - fy[:-2, :]) / (2 * h)


# ---------------------------------------------------------------------------
# Multidomain coupling (reading R5)
# ---------------------------------------------------------------------------

def _coarse_index(coord, origin, h):
    """Position of ``coord`` in units of the coarse spacing (a float)."""
    return (coord - origin) / h


def inject_fine_to_coarse(w_fine, fine, w_coarse, coarse):
    """Overwrite coarse vertices strictly inside ``fine`` by the coincident fine values."""
    xf, yf = fine.xv(), fine.yv()
    for jc, yc in enumerate(coarse.yv()):
        if not (yf[0] < yc < yf[-1]):
            continue
        jf = (yc - fine.y0) / fine.h
        jr = int(round(jf))
        assert abs(jf - jr) < 1e-9
        for ic, xc in enumerate(coarse.xv()):
            if not (xf[0] < xc < xf[-1]):
                continue
            i_f = (xc - fine.x0) / fine.h
            ir = int(round(i_f))
            assert abs(i_f - ir) < 1e-9
            w_coarse[jc, ic] = w_fine[jr, ir]


def interp_coarse_at(field_c, coarse, x, y):
    """Bilinear interpolation of a coarse vertex field at ``(x, y)`` (exact at coincident vertices)."""
    fi = _coarse_index(x, coarse.x0, coarse.h)
    fj = _coarse_index(y, coarse.y0, coarse.h)
    i0 = int(np.floor(fi + 1e-12))
    j0 = int(np.floor(fj + 1e-12))
    ti = fi - i0
    tj = fj - j0
    if abs(ti) < 1e-12:
        ti = 0.0
    if abs(tj) < 1e-12:
        tj = 0.0
    i1 = i0 + (1 if ti > 0 else 0)
    j1 = j0 + (1 if tj > 0 else 0)
    return ((1 - ti) * (1 - tj) * field_c[j0, i0] + ti * (1 - tj) * field_c[j0, i1]
            + (1 - ti) * tj * field_c[j1, i0] + ti * tj * field_c[j1, i1])


def set_ring_from_coarse(field_f, fine, field_c, coarse):
    """Boundary ring of the fine level from the coarse level (injection / midpoint averaging)."""
    xs, ys = fine.xv(), fine.yv()
    ny, nx = fine.ny, fine.nx
    for i in range(nx + 1):
        field_f[0, i] = interp_coarse_at(field_c, coarse, xs[i], ys[0])
        field_f[ny, i] = interp_coarse_at(field_c, coarse, xs[i], ys[ny])
    for j in range(1, ny):
        field_f[j, 0] = interp_coarse_at(field_c, coarse, xs[0], ys[j])
        field_f[j, nx] = interp_coarse_at(field_c, coarse, xs[nx], ys[j])
