"""Oracle: immersed-boundary coupling operators (FP64, numpy).

Test infrastructure only (see ``oracle/__init__.py``).

* ``delta3``     -- the 3-point regularised discrete delta (reading R1: Roma,
                    Peskin & Berger); the paper names no specific kernel (Sec. 3.1).
* ``hat``        -- the two-point hat ``d_p`` of Sec. 3.1.2 used to build ``P``
                    (``d_p = 0`` at ``|r| = dr``, reading R9).
* ``Subdomain``  -- the fixed sub-domain Omega_0: a box of flow-grid vertices at
                    spacing h (Sec. 3.1.1), and the operators
                    ``E0`` (Eq. ibsdinterp), ``E0^T`` and ``P`` (Eq. weights).
* ``b0_column``  -- column j of ``B0 = E0 C (C^T A C)^{-1} C^T E0^T`` computed as the
                    action on the canonical vector e_j (Eq. action, Algorithm 1), optionally
                    filtered by the drop tolerance of Eq. filtereq (``drop_filter``).
* ``e_points``, ``et_points``, ``ke_column`` -- the true IB interpolation ``E`` at the body
                    points themselves (Sec. 2.2, the operator the sub-domain approach replaces),
                    its transpose, and a column of ``E C (C^T A C)^{-1} C^T E^T``.

Unknown ordering of sub-domain vectors: the ``n_sd`` x-components first, then
the ``n_sd`` y-components; points are numbered row by row (j-major) inside the box.
"""

import numpy as np

from . import grid


def delta3(r):
    """3-point discrete delta in grid units (reading R1)."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    m1 = r <= 0.5
    out[m1] = (1.0 + np.sqrt(1.0 - 3.0 * r[m1] ** 2)) / 3.0
    m2 = (r > 0.5) & (r <= 1.5)
    out[m2] = (5.0 - 3.0 * r[m2] - np.sqrt(np.maximum(0.0, 1.0 - 3.0 * (1.0 - r[m2]) ** 2))) / 6.0
    return out


def hat(r, dr):
    """Two-point hat of Sec. 3.1.2: ``1 - |r|/dr`` for ``|r| < dr``, else 0."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    return np.where(r < dr, 1.0 - r / dr, 0.0)


class Subdomain:
    """Omega_0: the vertices ``i_lo..i_hi`` x ``j_lo..j_hi`` of the finest level (Sec. 3.1.1) -- or a union of
    such vertex boxes (reading R16: one box per body, the cross-box blocks of B0 included) -- followed by
    ``extra`` appended points, the exact points of stationary bodies, interpolated with E itself (Sec. 3.1.1:
    such points may be added to the sub-domain with weight one).  Unknowns: the x components of the ``n_box``
    box vertices (box by box, row by row inside a box) and of the extra points, then the y components
    likewise."""

    def __init__(self, lev, i_lo, i_hi, j_lo, j_hi, extra=None, boxes=None):
        boxes = [(i_lo, i_hi, j_lo, j_hi)] if boxes is None else [tuple(int(v) for v in b) for b in boxes]
        for (a, b, c, d) in boxes:
            if a < 2 or c < 2 or b > lev.nx - 2 or d > lev.ny - 2 or b <= a or d <= c:
                raise ValueError("sub-domain must lie at least 2 cells inside the grid")
        for k, (a, b, c, d) in enumerate(boxes):
            for (a2, b2, c2, d2) in boxes[:k]:
                if a <= b2 and a2 <= b and c <= d2 and c2 <= d:
                    raise ValueError("sub-domain boxes must not share vertices")
        self.lev = lev
        self.boxes = boxes
        self.i_lo, self.i_hi, self.j_lo, self.j_hi = boxes[0]
        self.ni = self.i_hi - self.i_lo + 1
        self.nj = self.j_hi - self.j_lo + 1
        pis, pjs, self.box_off = [], [], []
        for (a, b, c, d) in boxes:
            self.box_off.append(sum(len(x) for x in pis))
            jj, ii = np.meshgrid(np.arange(c, d + 1), np.arange(a, b + 1), indexing="ij")
            pis.append(ii.ravel())
            pjs.append(jj.ravel())
        self.pi = np.concatenate(pis)
        self.pj = np.concatenate(pjs)
        self.n_box = len(self.pi)
        self.extra = np.zeros((0, 2)) if extra is None else np.asarray(extra, dtype=np.float64).reshape(-1, 2)
        self.n_sd = self.n_box + len(self.extra)

    @staticmethod
    def _snap(lev, x_lo, x_hi, y_lo, y_hi):
        """Snap a physical box to vertices, clipped to >= 2 cells from the boundary (reading R10)."""
        i_lo = max(int(np.ceil((x_lo - lev.x0) / lev.h - 1e-9)), 2)
        i_hi = min(int(np.floor((x_hi - lev.x0) / lev.h + 1e-9)), lev.nx - 2)
        j_lo = max(int(np.ceil((y_lo - lev.y0) / lev.h - 1e-9)), 2)
        j_hi = min(int(np.floor((y_hi - lev.y0) / lev.h + 1e-9)), lev.ny - 2)
        return i_lo, i_hi, j_lo, j_hi

    @classmethod
    def from_box(cls, lev, x_lo, x_hi, y_lo, y_hi, extra=None):
        return cls(lev, *cls._snap(lev, x_lo, x_hi, y_lo, y_hi), extra)

    @classmethod
    def from_boxes(cls, lev, boxes, extra=None):
        """The union of several physical boxes, each snapped as ``from_box`` (reading R16)."""
        snapped = [cls._snap(lev, *b) for b in boxes]
        return cls(lev, *snapped[0], extra, boxes=snapped)

    # -- E0 (Eq. ibsdinterp): weights d(x_face - x_k) d(y_face - y_k) --------------------

    def _u_window(self):
        """u-face indices and delta weights around every Omega_0 point (support window, zeros kept)."""
        di = np.arange(-2, 3)
        dj = np.arange(-2, 2)             # u[j', i'] sits at y_{j'+1/2}
        I = self.pi[:, None, None] + di[None, None, :]
        J = self.pj[:, None, None] + dj[None, :, None]
        w = delta3(I - self.pi[:, None, None]) * delta3(J + 0.5 - self.pj[:, None, None])
        return I, J, w

    def _v_window(self):
        di = np.arange(-2, 2)             # v[j', i'] sits at x_{i'+1/2}
        dj = np.arange(-2, 3)
        I = self.pi[:, None, None] + di[None, None, :]
        J = self.pj[:, None, None] + dj[None, :, None]
        w = delta3(I + 0.5 - self.pi[:, None, None]) * delta3(J - self.pj[:, None, None])
        return I, J, w

    def e0(self, u, v):
        """``E0 q``: interpolate face fluxes to all Omega_0 points -> vector of length ``2 n_sd`` (E itself
        at the appended points)."""
        I, J, w = self._u_window()
        u0 = np.sum(w * u[J, I], axis=(1, 2))
        I, J, w = self._v_window()
        v0 = np.sum(w * v[J, I], axis=(1, 2))
        nx_ = len(self.extra)
        ex = e_points(self.lev, self.extra, u, v) if nx_ else np.zeros(0)
        return np.concatenate([u0, ex[:nx_], v0, ex[nx_:]])

    def e0t(self, g):
        """``E0^T g``: spread a sub-domain vector onto the faces (same weights, transposed)."""
        lev = self.lev
        nb_, n = self.n_box, self.n_sd
        u = np.zeros((lev.ny, lev.nx + 1))
        v = np.zeros((lev.ny + 1, lev.nx))
        I, J, w = self._u_window()
        np.add.at(u, (J, I), w * g[:nb_, None, None])
        I, J, w = self._v_window()
        np.add.at(v, (J, I), w * g[n:n + nb_, None, None])
        if len(self.extra):
            ue, ve = et_points(lev, self.extra, np.concatenate([g[nb_:n], g[n + nb_:]]))
            u += ue
            v += ve
        return u, v

    # -- P (Eqs. sdapprox3, weights): 4 tensor-cell neighbours, hat weights --------------

    def p_rows(self, pts, appended=None):
        """For each body point: the 4 Omega_0 point indices and hat weights (reading R9).  A point with
        ``appended[p] = e >= 0`` is extra point e itself: index n_box + e with weight one (the others zero)."""
        lev = self.lev
        if appended is not None and np.any(np.asarray(appended) >= 0):
            app = np.asarray(appended)
            idx = np.zeros((len(pts), 4), dtype=np.int64)
            wts = np.zeros((len(pts), 4))
            box = np.nonzero(app < 0)[0]
            if len(box):
                bi, bw = self.p_rows(np.asarray(pts)[box])
                idx[box], wts[box] = bi, bw
            for p in np.nonzero(app >= 0)[0]:
                idx[p, :] = self.n_box + app[p]
                wts[p, 0] = 1.0
            return idx, wts
        idx = np.zeros((len(pts), 4), dtype=np.int64)
        wts = np.zeros((len(pts), 4))
        for p, (x, y) in enumerate(pts):
            for (i_lo, i_hi, j_lo, j_hi), off in zip(self.boxes, self.box_off):   # the first box holding it
                x_lo, y_lo = lev.x0 + i_lo * lev.h, lev.y0 + j_lo * lev.h
                x_hi, y_hi = lev.x0 + i_hi * lev.h, lev.y0 + j_hi * lev.h
                if x_lo <= x <= x_hi and y_lo <= y <= y_hi:
                    break
            else:
                raise ValueError("body point outside the sub-domain")
            ni, nj = i_hi - i_lo + 1, j_hi - j_lo + 1
            ci = min(max(int(np.floor((x - x_lo) / lev.h)), 0), ni - 2)
            cj = min(max(int(np.floor((y - y_lo) / lev.h)), 0), nj - 2)
            k = 0
            for b in (0, 1):
                for a in (0, 1):
                    xs = x_lo + (ci + a) * lev.h
                    ys = y_lo + (cj + b) * lev.h
                    idx[p, k] = off + (cj + b) * ni + (ci + a)
                    wts[p, k] = hat(x - xs, lev.h) * hat(y - ys, lev.h)
                    k += 1
        return idx, wts


def drop_filter(b, col, drop_tol):
    """Eq. filtereq applied to column ``col`` as it is built (Algorithm 1): keep ``b_i`` where
    ``|b_i| > drop_tol |b_col|`` (the column's own diagonal, strict inequality: reading R8), else 0."""
    if drop_tol <= 0.0:
        return b
    return np.where(np.abs(b) > drop_tol * abs(b[col]), b, 0.0)


def b0_column(sd, col, re, dt, drop_tol=0.0):
    """Column ``col`` of ``B0``: ``E0 C Lap^{-1} A_w^{-1} C^T E0^T e_col`` (Eq. action), filtered by
    ``drop_filter`` when ``drop_tol > 0`` (the sparse ``B0'`` of Eq. filtereq).

    The solves use the finest level with homogeneous boundary values (reading R6).
    """
    lev = sd.lev
    e = np.zeros(2 * sd.n_sd)
    e[col] = 1.0
    u, v = sd.e0t(e)
    src = grid.curl_faces(u, v, lev)
    zero = np.zeros(lev.shape)
    w = grid.solve_aw(src, zero, lev, re, dt)
    s = np.zeros(lev.shape)
    s[1:-1, 1:-1] = grid.solve_lap(w, zero, lev)
    qu, qv = grid.faces_from_s(s, lev)
    return drop_filter(sd.e0(qu, qv), col, drop_tol)


def b0_dense(sd, re, dt):
    """All columns of ``B0`` (Algorithm 1 with zero drop tolerance); small grids only."""
    return np.stack([b0_column(sd, c, re, dt) for c in range(2 * sd.n_sd)], axis=1)


# -- true E at the body points (Sec. 2.2; the comparator of Sec. 5.1) ---------------------------

def _face_weights(lev, pts, comp):
    """Face indices and delta weights of every body point: u faces sit at (x_i, y_{j+1/2}), v faces at
    (x_{i+1/2}, y_j); the 3-point delta reaches 1.5 cells, so 4 x 4 candidate faces per point."""
    X = (np.asarray(pts)[:, 0] - lev.x0) / lev.h
    Y = (np.asarray(pts)[:, 1] - lev.y0) / lev.h
    ox, oy = (0.0, 0.5) if comp == 0 else (0.5, 0.0)
    i0 = np.floor(X - ox).astype(np.int64) - 1
    j0 = np.floor(Y - oy).astype(np.int64) - 1
    d = np.arange(4)
    I = i0[:, None, None] + d[None, None, :]
    J = j0[:, None, None] + d[None, :, None]
    w = delta3(I + ox - X[:, None, None]) * delta3(J + oy - Y[:, None, None])
    return I, J, w


def e_points(lev, pts, u, v):
    """``E q``: the face fluxes interpolated to the body points, (x components, then y components)."""
    I, J, w = _face_weights(lev, pts, 0)
    ub = np.sum(w * u[J, I], axis=(1, 2))
    I, J, w = _face_weights(lev, pts, 1)
    vb = np.sum(w * v[J, I], axis=(1, 2))
    return np.concatenate([ub, vb])


def et_points(lev, pts, f):
    """``E^T f``: a body-point vector spread onto the faces (same weights, transposed)."""
    nb = len(pts)
    u = np.zeros((lev.ny, lev.nx + 1))
    v = np.zeros((lev.ny + 1, lev.nx))
    I, J, w = _face_weights(lev, pts, 0)
    np.add.at(u, (J, I), w * np.asarray(f)[:nb, None, None])
    I, J, w = _face_weights(lev, pts, 1)
    np.add.at(v, (J, I), w * np.asarray(f)[nb:, None, None])
    return u, v


def ke_column(lev, pts, col, re, dt):
    """Column ``col`` of ``E C Lap^{-1} A_w^{-1} C^T E^T`` at the body points (the finest level with
    homogeneous boundary values, reading R6)."""
    e = np.zeros(2 * len(pts))
    e[col] = 1.0
    u, v = et_points(lev, pts, e)
    src = grid.curl_faces(u, v, lev)
    zero = np.zeros(lev.shape)
    w = grid.solve_aw(src, zero, lev, re, dt)
    s = np.zeros(lev.shape)
    s[1:-1, 1:-1] = grid.solve_lap(w, zero, lev)
    qu, qv = grid.faces_from_s(s, lev)
    return e_points(lev, pts, qu, qv)
