"""Pins for the oracle's multidomain level coupling (Sec. 5 intro: the far-field
scheme of Colonius & Taira; reading R5) with a Lamb-Oseen vortex.

The Lamb-Oseen vortex is an exact solution of the incompressible Navier-Stokes
equations: w(r, t) = Gamma / (4 pi nu t) exp(-r^2 / (4 nu t)) with nu = 1/Re.
Its velocity is azimuthal and its vorticity radial, so the advection term
vanishes and the vortex only diffuses.  Centred in the finest level with no
body and no free stream, it pins three things of the oracle's step that no
single-level test can see:

* far field -- the vortex extends past the finest level, so one level with
  zero boundary values is wrong by the cut-off tail; with a coarser level
  around it the error falls to the discretisation error (error vs G);
* the time level of the boundary values -- Crank-Nicolson with AB2 is second
  order in time only if each finer level takes its boundary w, s from the
  coarser level at t^{n+1}, i.e. the sweep runs coarse to fine; boundary
  values lagging by one step (a fine-to-coarse sweep, or rings set before the
  coarse solve) make the scheme first order;
* the fine-to-coarse injection -- it must replace the coarse vorticity inside
  the finer level before the coarse right-hand side is formed, so that the
  coarse level carries the fine level's accuracy there; injected after the
  right-hand side it has no effect and the coarse level keeps its own,
  four times larger, second-order error.

Each mistake is planted in a copy of the oracle's predictor (below, on the
CPU) to show that the test that pins it fails for it.  Errors are relative to
the peak vorticity at the final time.
"""

import numpy as np

from oracle import fsi, grid

GAMMA = 1.0
RE = 50.0
T0, T1 = 0.5, 1.0     # vortex core sqrt(4 nu t) = 0.2 -> 0.28; the finest level is [-0.5, 0.5]^2


def omega_exact(x, y, t, re=RE):
    nu = 1.0 / re
    return GAMMA / (4.0 * np.pi * nu * t) * np.exp(-(x * x + y * y) / (4.0 * nu * t))


def _start(sim, t0):
    """Exact vertex vorticity at t0 on every level's interior (the coarsest ring stays 0, as in a
    run); s from w coarse to fine with each finer ring taken from the coarser level."""
    G = len(sim.levels)
    for g, lev in enumerate(sim.levels):
        x, y = np.meshgrid(lev.xv(), lev.yv())
        sim.w[g][1:-1, 1:-1] = omega_exact(x, y, t0)[1:-1, 1:-1]
    for g in range(G - 1, -1, -1):
        if g < G - 1:
            grid.set_ring_from_coarse(sim.w[g], sim.levels[g], sim.w[g + 1], sim.levels[g + 1])
            grid.set_ring_from_coarse(sim.s[g], sim.levels[g], sim.s[g + 1], sim.levels[g + 1])
        sim.s[g][1:-1, 1:-1] = grid.solve_lap(sim.w[g][1:-1, 1:-1], sim.s[g], sim.levels[g])


def _run(nx, n_levels, dt, cls=fsi.Sim, half=0.5, t0=T0, t1=T1):
    h = 2.0 * half / nx
    sim = cls(nx, nx, h, -half, -half, n_levels, RE, dt, (0.0, 0.0), None, [], h)
    _start(sim, t0)
    for _ in range(int(round((t1 - t0) / dt))):
        sim.step()
    return sim


def _level_error(sim, g, mask=None, t=T1):
    """Max |w - exact| over level g's interior vertices (optionally masked), over the peak."""
    lev = sim.levels[g]
    x, y = np.meshgrid(lev.xv(), lev.yv())
    ex = omega_exact(x, y, t)
    err = np.abs(sim.w[g] - ex)[1:-1, 1:-1]
    if mask is not None:
        err = err[mask[1:-1, 1:-1]]
    return float(np.max(err)) / omega_exact(0.0, 0.0, t)


# ------------------------------------------------------------------ planted mistakes (CPU)

def _rhs_all(sim):
    L, dt, re = sim.levels, sim.dt, sim.re
    rhs = []
    for g in range(len(L)):
        n_now = grid.nonlinear(sim.s[g], sim.w[g], L[g], sim.uinf)
        n_old = n_now if sim.nprev[g] is None else sim.nprev[g]
        rhs.append(sim.w[g][1:-1, 1:-1] / dt + grid.laplacian(sim.w[g], L[g]) / (2.0 * re)
                   - 1.5 * n_now + 0.5 * n_old)
        sim.nprev[g] = n_now
    return rhs


def _solve_level(sim, g, r):
    lev = sim.levels[g]
    w_int = grid.solve_aw(r, sim.w[g], lev, sim.re, sim.dt)
    sim.w[g][1:-1, 1:-1] = w_int
    sim.s[g][1:-1, 1:-1] = grid.solve_lap(w_int, sim.s[g], lev)


def _ring(sim, g):
    L = sim.levels
    grid.set_ring_from_coarse(sim.w[g], L[g], sim.w[g + 1], L[g + 1])
    grid.set_ring_from_coarse(sim.s[g], L[g], sim.s[g + 1], L[g + 1])


class FineToCoarseSweep(fsi.Sim):
    """Mistake: levels solved fine to coarse, so every ring comes from the coarser level at t^n."""

    def predictor(self):
        G = len(self.levels)
        for g in range(G - 1):
            grid.inject_fine_to_coarse(self.w[g], self.levels[g], self.w[g + 1], self.levels[g + 1])
        rhs = _rhs_all(self)
        for g in range(G):
            if g < G - 1:
                _ring(self, g)
            _solve_level(self, g, rhs[g])


class RingsBeforeSolves(fsi.Sim):
    """Mistake: coarse to fine, but every ring is set before any level is solved (rings at t^n)."""

    def predictor(self):
        G = len(self.levels)
        for g in range(G - 1):
            grid.inject_fine_to_coarse(self.w[g], self.levels[g], self.w[g + 1], self.levels[g + 1])
        rhs = _rhs_all(self)
        for g in range(G - 2, -1, -1):
            _ring(self, g)
        for g in range(G - 1, -1, -1):
            _solve_level(self, g, rhs[g])


class InjectionAfterRhs(fsi.Sim):
    """Mistake: the fine-to-coarse injection comes after the right-hand sides are formed."""

    def predictor(self):
        G = len(self.levels)
        rhs = _rhs_all(self)
        for g in range(G - 1):
            grid.inject_fine_to_coarse(self.w[g], self.levels[g], self.w[g + 1], self.levels[g + 1])
        for g in range(G - 1, -1, -1):
            if g < G - 1:
                _ring(self, g)
            _solve_level(self, g, rhs[g])


def _time_order(cls):
    """Observed order in dt at fixed grid from three runs at dt, dt/2, dt/4 (successive differences)."""
    ws = [_run(32, 2, dt, cls).w[0] for dt in (0.02, 0.01, 0.005)]
    d1 = np.max(np.abs(ws[0] - ws[1]))
    d2 = np.max(np.abs(ws[1] - ws[2]))
    return float(np.log2(d1 / d2))


# ------------------------------------------------------------------ pins

def test_lamb_oseen_error_falls_with_levels():
    """One level cuts the vortex off at the finest boundary (about 4 % of the peak there at T1);
    a second level around it brings the error down to the discretisation error, a third keeps it."""
    errs = [_level_error(_run(32, G, 0.01), 0) for G in (1, 2, 3)]
    assert errs[0] > 5.0 * errs[1], errs
    assert errs[2] <= 1.01 * errs[1], errs
    assert errs[1] < 5e-3, errs


def test_lamb_oseen_second_order_in_space():
    """Three levels, finest h = 1/32 and 1/64 with dt proportional to h: the finest-level error
    falls at second order (5-point stencils, Crank-Nicolson, central advection)."""
    e32 = _level_error(_run(32, 3, 0.01), 0)
    e64 = _level_error(_run(64, 3, 0.005), 0)
    order = np.log2(e32 / e64)
    assert 1.8 < order < 2.2, (e32, e64, order)


def test_lamb_oseen_second_order_in_time_needs_rings_at_new_time():
    """At a fixed grid the two-level solution converges at second order in dt; boundary values taken
    at t^n (fine-to-coarse sweep, or rings set before the coarse solve) drop it to first order."""
    good = _time_order(fsi.Sim)
    assert 1.9 < good < 2.1, good
    for cls in (FineToCoarseSweep, RingsBeforeSolves):
        bad = _time_order(cls)
        assert bad < 1.3, (cls.__name__, bad)


def test_injection_gives_the_coarse_level_fine_accuracy_inside():
    """Inside the finer level the coarse vorticity is the injected fine one (advanced by one coarse
    step), so its error is close to the fine level's; without an effective injection it is the coarse
    level's own second-order error, about four times larger."""
    def errors(cls):
        sim = _run(32, 2, 0.01, cls)
        lev = sim.levels[1]
        x, y = np.meshgrid(lev.xv(), lev.yv())
        inside = (np.abs(x) < 0.5 - 1e-12) & (np.abs(y) < 0.5 - 1e-12)
        return _level_error(sim, 0), _level_error(sim, 1, inside)

    fine, coarse_in = errors(fsi.Sim)
    assert coarse_in < 1.2 * fine, (fine, coarse_in)
    fine_bad, coarse_in_bad = errors(InjectionAfterRhs)
    assert coarse_in_bad > 3.0 * fine_bad, (fine_bad, coarse_in_bad)


def test_fine_ring_holds_the_coarse_level_at_the_same_time():
    """After every step of a correct sweep, the finer level's ring equals the coarser level's field at
    the same time (injection at coincident vertices, midpoint averages between): exact to rounding.
    The fine-to-coarse sweep leaves the ring one step behind and fails it."""
    def max_ring_gap(cls, steps=4):
        sim = _run(32, 3, 0.01, cls, t1=T0 + steps * 0.01)
        gap = 0.0
        for g in range(len(sim.levels) - 1):
            for field in (sim.w, sim.s):
                ref = field[g].copy()
                grid.set_ring_from_coarse(ref, sim.levels[g], field[g + 1], sim.levels[g + 1])
                gap = max(gap, float(np.max(np.abs(ref - field[g]))) / float(np.max(np.abs(field[g]))))
        return gap

    assert max_ring_gap(fsi.Sim) < 1e-14
    assert max_ring_gap(FineToCoarseSweep) > 1e-6
