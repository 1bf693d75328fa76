"""FP64 CPU oracle for the sub-domain strongly coupled immersed-boundary FSI method
(Nair & Goza, "A strongly coupled immersed boundary method for fluid-structure
interaction that mimics the efficiency of stationary body methods").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library.

Everything is plain numpy in float64.  The one library primitive used for a
transform is a dense matrix product with the sine matrix (a naive O(N^2)
DST-I per axis).  Small dense systems are solved with ``numpy.linalg.solve``.

Module map
  grid.py  -- staggered streamfunction/vorticity operators, DST-diagonalised
              solves, nested multidomain levels (Sec. 2.2, Sec. 3.2.1, App. A)
  ib.py    -- discrete delta, sub-domain interpolation E0, hat interpolation P,
              sub-domain matrix B0 by columns (Sec. 3.1, Eqs. ibsdinterp,
              weights, action; Algorithm 1)
  fsi.py   -- torsional / rigid bodies, FSI iteration, one time step and runs
              (Eqs. predictor2-corrector2, Algorithm 2, App. A)
  beam.py  -- deformable flag: corotational Euler-Bernoulli beam, lumped mass,
              trapezoidal Newmark (Sec. 2.1 Eq. beam, App. A)
  kinematics.py -- prescribed heave/pitch of a driven plate and the passive plate hinged to it
              (Sec. 5.1, Eq. newtonseldg)

Parity status: every function here is pinned by ``tests/test_oracle_*.py``.
The multidomain level coupling is pinned by a Lamb-Oseen vortex
(``tests/test_oracle_multidomain.py``): error against the closed form falling
with the number of levels and at second order in h and in dt, the coarse level
carrying the fine level's accuracy inside it, and the finer rings holding the
coarser level at the same time; each of those fails for a planted wrong sweep
order, ring time level or injection order.
"""

from . import grid, ib, fsi, beam, kinematics  # noqa: F401
