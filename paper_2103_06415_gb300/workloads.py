"""Synthetic workloads shaped like the paper's experiments, and seeded input generators.

This module holds parameters and random inputs only (no arithmetic of the method), so both the CUDA
path and the CPU oracle can be driven from the same inputs.

Configurations:

* ``plate_128``  -- single level 128x128 cells on [-1,3]x[-2,2] (h = 1/32), Re 100, dt 0.002, one rigid
  flat plate of chord 1 hinged at its leading edge (0,0) on a torsional spring (inertia 1, stiffness 0.5,
  no damping), initial angle 20 deg, 33 points at ds = h; Omega_0 = [-1.2,1.2]^2.
* ``plate_128_ds2h`` -- plate_128 with 17 points at ds = 2h (the paper's body spacing).
* ``e1_flapping`` -- the flapping torsionally connected plates of Sec. 5.1 (cases 1, 2 of Table kineparams)
  on 5 levels of 512 x 512; ``small_flapping`` the same pair on a 64 x 64 grid.
* ``flag_512x256_3lvl`` -- 3 nested levels of 512x256 cells, finest h = 1/100 on [-1,4.12]x[-1.28,1.28],
  Re 200, dt 5e-4; body: a flag of length 1 clamped at (0,0) along +x, 101 points (100 beam elements at
  ds = h), mass ratio 0.1, bending stiffness 1e-3, stretching stiffness 1e3, initial tip slope 0.1 rad;
  Omega_0 = [-0.2,1.2]x[-0.7,0.7] (141 x 141 points).
* ``flag_512x256_3lvl_torsional`` -- the same grid with a torsional plate of 101 points standing in for
  the flag (inertia 0.1/3, spring 1e-3, initial angle 0.1 rad).
"""

import numpy as np

SEED = 20261203


def plate_128():
    return dict(
        name="plate_128", nx=128, ny=128, n_levels=1, x0=-1.0, y0=-2.0, h=1.0 / 32, re=100.0, dt=0.002,
        uinf=(1.0, 0.0), steps=100, sd_box=(-1.2, 1.2, -1.2, 1.2),
        bodies=[dict(kind="torsional", hinge=(0.0, 0.0), theta0=0.0, n_pts=33, inertia=1.0, damping=0.0,
                     stiffness=0.5, theta=np.deg2rad(20.0))],
        ds=1.0 / 32)


def plate_128_ds2h():
    """plate_128 with the body points at twice the grid spacing, the paper's choice for its experiments
    (Sec. 5): 17 points at ds = 2h = 1/16 on the same chord."""
    w = plate_128()
    w["name"] = "plate_128_ds2h"
    w["bodies"][0]["n_pts"] = 17
    w["ds"] = 2.0 / 32
    return w


def flag_512x256_3lvl():
    return dict(
        name="flag_512x256_3lvl", nx=512, ny=256, n_levels=3, x0=-1.0, y0=-1.28, h=0.01, re=200.0, dt=5e-4,
        uinf=(1.0, 0.0), steps=2000, sd_box=(-0.2, 1.2, -0.7, 0.7),
        bodies=[dict(kind="deformable", clamp=(0.0, 0.0), theta0=0.0, n_pts=101, mass=0.1, ei=1e-3, ea=1e3,
                     tip_angle=0.1)],
        ds=0.01)


def flag_512x256_3lvl_torsional():
    w = flag_512x256_3lvl()
    w["name"] = "flag_512x256_3lvl_torsional"
    w["bodies"] = [dict(kind="torsional", hinge=(0.0, 0.0), theta0=0.0, n_pts=101, inertia=0.1 / 3.0, damping=0.0,
                        stiffness=1e-3, theta=0.1)]
    return w


def _flapping_pair(n_pts, ds, a0, beta, sigma_t, sigma_r, theta=0.0):
    """Driven plate (reference point at the origin, from 0.5 above it to the hinge 0.55 below it at
    alpha1 = 0) and the passive plate hinged at its end (Sec. 5.1): both 1.05 long, n_pts - 1 segments of
    ds.  The hinge point is kept once, on the passive plate (two coincident points would make two rows of
    the interpolation equal and the small system singular), so the driven plate has n_pts - 1 points; passive plate of
    mass pi/4 (density ratio 5 for the 5:1 ellipse of unit chord), moment of inertia 0.2886 about the
    hinge, centre of mass 0.55 from the hinge, spring 456, damper 3.95 (all made dimensionless with
    the flapping frequency f and the chord)."""
    return [dict(kind="driven", ref=(0.0, 0.0), s_lo=-0.5, n_pts=n_pts - 1, a0=a0, beta=beta, sigma_t=sigma_t,
                 sigma_r=sigma_r, freq=1.0),
            dict(kind="hinged", driver=0, l1=0.55, n_pts=n_pts, inertia=0.2886, damping=3.95, stiffness=456.0,
                 mass=np.pi / 4.0, l2=0.55, theta=theta)]


def e1_flapping(case=1):
    """Flapping of torsionally connected plates (Sec. 5.1, Table kineparams): A0 = 1.4, beta = pi/4,
    sigma_t = sigma_r = 3.770 (case 1) or 0.628 (case 2), Re_r = 100, so Re = f c^2 / nu
    = Re_r tanh(sigma_r) / (2 pi beta sigma_r); hovering (no free stream).  dt = 0.00489 tau_r of case 1
    (tau_r = tanh(sigma_r) / (2 pi beta sigma_r) periods; the ratio comes from the convergence study on
    case 1) for both cases: at case 2's own tau_r the step would be 3.3 times longer and the explicit
    advection of the fast passive tip exceeds its stability limit (CFL 2.2 before the run diverges).  Five levels of 512 x 512 cells over the paper's finest
    domain [-3.15, 3.15] x [-4.65, 1.65] (h = 0.0123; the paper's 600 x 600 at 0.0105 is not a power of
    two); Omega_0 = [-1.89, 1.89] x [-1.66, 0.65]; plates at ds = 1.05/43 (about 2h, the paper's body
    spacing): 43 driven points and 44 passive points (the hinge point on the passive plate)."""
    sig = 3.770 if case == 1 else 0.628
    beta = np.pi / 4.0
    tau_r = np.tanh(sig) / (2.0 * np.pi * beta * sig)
    dt = 0.00489 * np.tanh(3.770) / (2.0 * np.pi * beta * 3.770)
    h = 6.3 / 512
    return dict(name="e1_flapping_case%d" % case, nx=512, ny=512, n_levels=5, x0=-3.15, y0=-4.65, h=h,
                re=100.0 * tau_r, dt=dt, uinf=(0.0, 0.0), steps=int(round(1.0 / dt)),
                sd_box=(-1.89, 1.89, -1.66, 0.65), bodies=_flapping_pair(44, 1.05 / 43, 1.4, beta, sig, sig),
                ds=1.05 / 43, l1=0.55)


def small_flapping(a0=1.4, beta=np.pi / 4.0, sigma=0.628, dt=0.004):
    """The flapping pair on a 64 x 64 grid (h = 1/16) the oracle runs in seconds: 16 driven and 17 passive
    points."""
    h = 1.0 / 16
    tau_r = np.tanh(sigma) / (2.0 * np.pi * np.pi / 4.0 * sigma)
    return dict(name="small_flapping", nx=64, ny=64, n_levels=1, x0=-2.0, y0=-2.75, h=h, re=100.0 * tau_r, dt=dt,
                uinf=(0.0, 0.0), steps=10, sd_box=(-1.6, 1.6, -2.0, 0.7),
                bodies=_flapping_pair(17, 1.05 / 16, a0, beta, sigma, sigma), ds=1.05 / 16, l1=0.55)


def b0_1024():
    """Offline benchmark: B0 for a 64 x 64-vertex Omega_0 (4096 points, 8192 unknowns) centred in a
    1024 x 1024 grid, h = 1/256, Re 500, dt = h/4 (alpha = dt/(2 Re h^2) = 0.064); no bodies."""
    h = 1.0 / 256
    return dict(name="b0_1024", nx=1024, ny=1024, n_levels=1, x0=-2.0, y0=-2.0, h=h, re=500.0, dt=h / 4,
                uinf=(1.0, 0.0), steps=0, sd_box=(-32 * h, 31 * h, -32 * h, 31 * h), bodies=[], ds=h)


B0_UNEVEN_SIDES = (16, 19, 22, 25, 28, 32, 35, 38, 41, 44, 48, 51, 54, 57, 60, 64)


def b0_1024_uneven_boxes(sides=B0_UNEVEN_SIDES, n=1024):
    """Sixteen square Omega_0 boxes of side s points (256 ... 4096 points each) on the b0_1024 grid, one per
    cell of a 4 x 4 arrangement of the domain (box k centred in cell k), as (x_lo, x_hi, y_lo, y_hi)."""
    w = b0_1024() if n == 1024 else None
    h, x0, y0 = (w["h"], w["x0"], w["y0"]) if w else (1.0 / 256, -2.0, -2.0)
    cell = n // 4
    boxes = []
    for k, s in enumerate(sides):
        cx, cy = cell // 2 + cell * (k % 4), cell // 2 + cell * (k // 4)
        i_lo, j_lo = cx - s // 2, cy - s // 2
        boxes.append((x0 + i_lo * h, x0 + (i_lo + s - 1) * h, y0 + j_lo * h, y0 + (j_lo + s - 1) * h))
    return boxes


def flag_512x256_3lvl_reduced_omega0():
    """flag_512x256_3lvl with Omega_0 cut to [-0.2,1.2]x[-0.25,0.35] (141 x 61 points, B0 2.4 GB); same
    kernels and small-system size, for profiler captures that must hold only a few GB."""
    w = flag_512x256_3lvl()
    w["name"] = "flag_512x256_3lvl_reduced_omega0"
    w["sd_box"] = (-0.2, 1.2, -0.25, 0.35)
    return w


def small_plate(nx=64, ny=32, n_levels=1):
    """A small torsional-plate case the oracle runs in seconds (several FFT tiles, ragged Omega_0 box)."""
    h = 1.0 / 16
    return dict(
        name="small_plate_%dx%d_%dlvl" % (nx, ny, n_levels), nx=nx, ny=ny, n_levels=n_levels, x0=-1.0,
        y0=-1.0, h=h, re=100.0, dt=0.004, uinf=(1.0, 0.0), steps=20, sd_box=(-0.6, 0.8, -0.7, 0.8),
        bodies=[dict(kind="torsional", hinge=(0.0, 0.0), theta0=0.0, n_pts=9, inertia=0.05, damping=0.0,
                     stiffness=0.5, theta=np.deg2rad(20.0))],
        ds=h)


def small_flag(nx=64, ny=32, n_levels=1, n_pts=9, tip_angle=0.1):
    """A small clamped flag the oracle runs in seconds: length (n_pts - 1) h, mass ratio 0.1, bending
    stiffness 1e-3, stretching stiffness 1e3."""
    h = 1.0 / 16
    return dict(
        name="small_flag_%dx%d_%dlvl" % (nx, ny, n_levels), nx=nx, ny=ny, n_levels=n_levels, x0=-1.0, y0=-1.0,
        h=h, re=100.0, dt=0.004, uinf=(1.0, 0.0), steps=20, sd_box=(-0.6, 0.8, -0.7, 0.8),
        bodies=[dict(kind="deformable", clamp=(0.0, 0.0), theta0=0.0, n_pts=n_pts, mass=0.1, ei=1e-3, ea=1e3,
                     tip_angle=tip_angle)],
        ds=h)


def small_mixed_bodies():
    """Two flags and a torsional plate sharing one Omega_0 (body and element offsets all non-zero)."""
    w = small_flag(nx=64, ny=64)
    w["name"] = "small_mixed_bodies"
    w["y0"] = -2.0
    w["sd_box"] = (-0.6, 0.9, -1.0, 1.0)
    w["bodies"] = [
        dict(kind="deformable", clamp=(0.0, 0.55), theta0=0.2, n_pts=6, mass=0.2, ei=2e-3, ea=5e2, tip_angle=-0.05),
        dict(kind="torsional", hinge=(0.0, 0.0), theta0=0.0, n_pts=7, inertia=0.05, damping=0.0, stiffness=0.5,
             theta=np.deg2rad(15.0)),
        dict(kind="deformable", clamp=(0.0, -0.55), theta0=-0.1, n_pts=9, mass=0.1, ei=1e-3, ea=1e3, tip_angle=0.1),
    ]
    return w


def serving_grid(n, re=100.0):
    """Serving request grid: n x n cells at the fixed h = 1/32 and dt = 0.002 of plate_128, domain
    [-1, -1 + n/32] x [-n/64, n/64], Omega_0 = [-1.2, 1.2]^2 clipped."""
    h = 1.0 / 32
    return dict(name="serve_%d" % n, nx=n, ny=n, n_levels=1, x0=-1.0, y0=-n / 64.0, h=h, re=re, dt=0.002,
                uinf=(1.0, 0.0), sd_box=(-1.2, 1.2, -1.2, 1.2), ds=h)


def serving_requests(n_req, seed=SEED, sizes=(128, 256, 512, 1024), steps=(200, 2000), rate_hz=20.0):
    """Poisson-arrival stream of independent torsional-plate runs (the serving workload's distributions):
    grid from `sizes`, Re ~ U[50, 300], stiffness log-uniform [0.05, 5], inertia ~ U[0.5, 2], angle of
    attack ~ U[5, 40] deg, steps ~ U{steps}.  Returns [(arrival_s, grid dict, body dict, n_steps)]."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for _ in range(n_req):
        t += rng.exponential(1.0 / rate_hz)
        n = int(rng.choice(sizes))
        w = serving_grid(n, re=float(rng.uniform(50.0, 300.0)))
        body = dict(kind="torsional", hinge=(0.0, 0.0), theta0=0.0, n_pts=33,
                    inertia=float(rng.uniform(0.5, 2.0)), damping=0.0,
                    stiffness=float(np.exp(rng.uniform(np.log(0.05), np.log(5.0)))),
                    theta=float(np.deg2rad(rng.uniform(5.0, 40.0))))
        out.append((t, w, body, int(rng.integers(steps[0], steps[1] + 1))))
    return out


def random_field(shape, seed, smooth=True):
    """Seeded vertex field: a few low sine modes plus small noise (ring included)."""
    rng = np.random.default_rng(seed)
    ny1, nx1 = shape
    y = np.linspace(0, 1, ny1)[:, None]
    x = np.linspace(0, 1, nx1)[None, :]
    f = np.zeros(shape)
    if smooth:
        for _ in range(4):
            k, l = rng.integers(1, 5, size=2)
            f += rng.standard_normal() * np.sin(np.pi * k * x) * np.sin(np.pi * l * y)
    f += 0.05 * rng.standard_normal(shape)
    return f


def random_rhs(ny_int, nx_int, seed):
    return np.random.default_rng(seed).standard_normal((ny_int, nx_int))


def tandem_small(nx=96, ny=48, n_levels=2):
    """A small case shaped like the large coupled workload (5 levels of 1536 x 768): a grid of 3 * 2^k cells,
    two torsional plates in tandem and a clamped flag behind them, each inside its own Omega_0 box (the
    union of the three boxes, reading R16); h = 1/16 on [-1, 5] x [-1.5, 1.5], Re 100, dt 0.004, chords
    0.5 (9 points at ds = h), plate springs 0.5 and 2, flag mass ratio 0.5, bending stiffness 1e-2."""
    h = 1.0 / 16
    hinges = [(0.0, 0.0), (1.25, 0.0), (2.5, 0.0)]
    return dict(
        name="tandem_small_%dx%d_%dlvl" % (nx, ny, n_levels), nx=nx, ny=ny, n_levels=n_levels, x0=-1.0,
        y0=-ny * h / 2, h=h, re=100.0, dt=0.004, uinf=(1.0, 0.0), steps=20,
        sd_box=[(hx - 0.2, hx + 0.7, -0.6, 0.6) for hx, _ in hinges],
        bodies=[dict(kind="torsional", hinge=hinges[0], theta0=0.0, n_pts=9, inertia=0.05, damping=0.0,
                     stiffness=0.5, theta=np.deg2rad(20.0)),
                dict(kind="torsional", hinge=hinges[1], theta0=0.0, n_pts=9, inertia=0.05, damping=0.0,
                     stiffness=2.0, theta=np.deg2rad(20.0)),
                dict(kind="deformable", clamp=hinges[2], theta0=0.0, n_pts=9, mass=0.5, ei=1e-2, ea=1e3,
                     tip_angle=0.1)],
        ds=h)


def tandem_nf246():
    """Three bodies of 41 points (two torsional plates and a flag, chord 1.25 at ds = h = 1/32) in three
    Omega_0 boxes on 192 x 96 cells, 2 levels: nf = 246, beyond the small system the FSI kernel can hold in
    shared memory, so the distributed block-inverse solver runs; small enough for the oracle."""
    h = 1.0 / 32
    hinges = [(-0.6, 0.0), (1.2, 0.0), (3.0, 0.0)]
    return dict(
        name="tandem_nf246_192x96_2lvl", nx=192, ny=96, n_levels=2, x0=-1.0, y0=-1.5, h=h, re=100.0, dt=0.004,
        uinf=(1.0, 0.0), steps=20, sd_box=[(hx - 0.2, hx + 1.45, -0.7, 0.7) for hx, _ in hinges],
        bodies=[dict(kind="torsional", hinge=hinges[0], theta0=0.0, n_pts=41, inertia=0.5, damping=0.0,
                     stiffness=0.5, theta=np.deg2rad(15.0)),
                dict(kind="torsional", hinge=hinges[1], theta0=0.0, n_pts=41, inertia=0.5, damping=0.0,
                     stiffness=2.0, theta=np.deg2rad(15.0)),
                dict(kind="deformable", clamp=hinges[2], theta0=0.0, n_pts=41, mass=0.5, ei=1e-2, ea=1e3,
                     tip_angle=0.1)],
        ds=h)


def tandem_1536x768_5lvl():
    """The large coupled workload: 5 nested levels of 1536 x 768 cells, finest h = 1/200 on
    [-1, 6.68] x [-1.92, 1.92], Re 1000, dt 2e-4, 5000 steps; three torsionally hinged plates of chord 1
    (201 points at ds = h) in tandem, hinged at (0, 0), (1.5, 0), (3, 0), initial angle 20 degrees, springs
    0.2, 1 and 5 (inertia 1, no damping; the workload gives the springs only), and a clamped flag of length 1
    (201 points) at (4.5, 0) with mass ratio 1, bending stiffness 1e-4, stretching stiffness 1e3 and initial tip
    slope 0.1 rad; each body inside its own Omega_0 box [x_h - 0.1, x_h + 1.1] x [-1.1, 1.1] (241 x 441
    vertices, 425 k points in the union, 850 k unknowns), so B0 is the filtered B0' (Eq. filtereq, eps = 0.007;
    dense it would hold 5.8 TB).  nf = 1608."""
    h = 1.0 / 200
    hinges = [(0.0, 0.0), (1.5, 0.0), (3.0, 0.0), (4.5, 0.0)]
    plates = [dict(kind="torsional", hinge=hinges[k], theta0=0.0, n_pts=201, inertia=1.0, damping=0.0,
                   stiffness=kk, theta=np.deg2rad(20.0)) for k, kk in enumerate((0.2, 1.0, 5.0))]
    flag = dict(kind="deformable", clamp=hinges[3], theta0=0.0, n_pts=201, mass=1.0, ei=1e-4, ea=1e3, tip_angle=0.1)
    return dict(
        name="tandem_1536x768_5lvl", nx=1536, ny=768, n_levels=5, x0=-1.0, y0=-1.92, h=h, re=1000.0, dt=2e-4,
        uinf=(1.0, 0.0), steps=5000, sd_box=[(hx - 0.1, hx + 1.1, -1.1, 1.1) for hx, _ in hinges],
        bodies=plates + [flag], ds=h, drop_tol=0.007)


def tandem_1536x768_reduced():
    """tandem_1536x768_5lvl for profiler captures that must hold a few GB: the same bodies (nf = 1608) on the
    same finest grid with 2 levels and Omega_0 boxes cut to [-0.45, 0.45] in y (B0' ~3.5 GB instead of 10 GB)."""
    w = tandem_1536x768_5lvl()
    w["name"] = "tandem_1536x768_reduced"
    w["n_levels"] = 2
    w["sd_box"] = [(b[0], b[1], -0.45, 0.45) for b in w["sd_box"]]
    return w
