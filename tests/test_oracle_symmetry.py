"""Mirror-symmetry pins of the oracle's coupled step (CPU).

A grid symmetric about y = 0 (vertex rows at +-y alike, the staggered u faces mapped onto u faces and v onto
-v), a sub-domain box symmetric about y = 0 and a plate lying along y = 0 make the discrete problem of
Algorithm 2 invariant under the reflection y -> -y, which maps the vorticity to minus its mirror image and the
lift and hinge moment to their negatives.  So:

* with the free stream along x, the lift, the moment and the deflection stay zero to rounding and the
  vorticity is antisymmetric about y = 0;
* with the free stream turned by +a and -a, the two runs have the same drag and opposite lift and moment;
* the drag is positive: f is the force per unit length the fluid exerts on the body (reading R2), and the
  impulsively started stream pushes the plate downstream.

An index shifted in y breaks one of these (planted on the CPU: a vertex average of the u faces taken from
one row twice in the advection term, and the hat cell of points above the axis shifted by one row, each fail
the tests below).  Mistakes that the reflection maps onto themselves, such as a sign flipped in the y
component of the spreading or in the free stream's y component, leave the mirror images equal; the no-slip,
closed-form and brute-force pins cover those.
"""

import numpy as np

from oracle import fsi

H = 1.0 / 16
BOX = (-0.6, 0.8, -0.75, 0.75)       # vertex-aligned, symmetric about y = 0


def _run(uinf, n_steps=6):
    # 48 x 40 cells on [-1, 2] x [-1.25, 1.25]: vertex rows at -1.25 + j / 16, symmetric about y = 0
    body = fsi.TorsionalBody((0.0, 0.0), 0.0, 9, H, 1.0, 0.0, 0.5, 0.0)
    sim = fsi.Sim(48, 40, H, -1.0, -1.25, 1, 100.0, 0.004, uinf, BOX, [body], H)
    for _ in range(n_steps):
        sim.step()
    hist = np.array([[r["bodies"][0][k] for k in ("fx", "fy", "moment", "theta")] for r in sim.history])
    return sim, hist


def test_plate_along_the_stream_has_no_lift_and_an_antisymmetric_wake():
    sim, hist = _run((1.0, 0.0))
    fx, fy, mom, th = hist.T
    scale = np.max(np.abs(fx))
    assert np.all(fx > 0.0)                        # drag: the fluid pushes the plate downstream
    assert np.max(np.abs(fy)) < 1e-12 * scale
    assert np.max(np.abs(mom)) < 1e-12 * scale
    assert np.max(np.abs(th)) < 1e-14
    w = sim.w[0]
    assert np.max(np.abs(w + w[::-1, :])) < 1e-11 * np.max(np.abs(w))


def test_stream_turned_up_and_down_mirrors_lift_and_moment():
    a = np.deg2rad(6.0)
    _, up = _run((np.cos(a), np.sin(a)))
    _, down = _run((np.cos(a), -np.sin(a)))
    scale = np.max(np.abs(up[:, :3]))
    assert np.max(np.abs(up[:, 1])) > 1e-3 * scale  # the turned stream does lift the plate
    assert np.max(np.abs(up[:, 0] - down[:, 0])) < 1e-11 * scale
    assert np.max(np.abs(up[:, 1] + down[:, 1])) < 1e-11 * scale
    assert np.max(np.abs(up[:, 2] + down[:, 2])) < 1e-11 * scale
    assert np.max(np.abs(up[:, 3] + down[:, 3])) < 1e-11 * max(np.max(np.abs(up[:, 3])), 1e-300)


def _run_flag(tip_angle, n_steps=6):
    from oracle import beam
    flag = beam.Beam((0.0, 0.0), 0.0, 8, H, 0.1, 1e-3, 1e3, tip_angle=tip_angle)
    sim = fsi.Sim(48, 40, H, -1.0, -1.25, 1, 100.0, 0.004, (1.0, 0.0), BOX, [flag], H)
    for _ in range(n_steps):
        sim.step()
    return sim, np.array([[r["bodies"][0][k] for k in ("fx", "fy", "theta")] for r in sim.history])


def test_flag_started_up_and_down_mirrors_lift_and_tip():
    """The deformable body (reading R18) under the same reflection: a flag along the stream with no initial
    bend keeps no lift and no tip deflection, and flags started with tip slopes +-0.1 rad have equal drag and
    opposite lift and tip deflection."""
    _, flat = _run_flag(0.0)
    scale = np.max(np.abs(flat[:, 0]))   # (the light flag's drag oscillates after the impulsive start)
    assert np.max(np.abs(flat[:, 1])) < 1e-12 * scale
    assert np.max(np.abs(flat[:, 2])) < 1e-14
    _, up = _run_flag(0.1)
    _, down = _run_flag(-0.1)
    assert np.max(np.abs(up[:, 2])) > 1e-3                      # the bent flag's tip is off the axis
    assert np.max(np.abs(up[:, 0] - down[:, 0])) < 1e-11 * scale
    assert np.max(np.abs(up[:, 1] + down[:, 1])) < 1e-11 * scale
    assert np.max(np.abs(up[:, 2] + down[:, 2])) < 1e-11 * np.max(np.abs(up[:, 2]))
