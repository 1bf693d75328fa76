"""The headline workload at full size (3 levels of 512 x 256, the 101-point flag, Omega_0 141 x 141, 39 762
unknowns) against the oracle on what it can compute one by one: sampled columns of B0, and the no-slip
identity after the corrector, which holds at any size (needs a GB300 and the library)."""

import numpy as np
import pytest

from oracle import grid as og
from oracle import ib as oib
from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


@pytest.fixture(scope="module")
def setup():
    w = wl.flag_512x256_3lvl()
    lev = og.make_levels(w["nx"], w["ny"], w["h"], w["x0"], w["y0"], w["n_levels"])[0]
    sd = oib.Subdomain.from_box(lev, *w["sd_box"])
    return w, lev, sd


def test_sampled_b0_columns_at_full_size(lib, setup):
    """B0 of the bench's FP32 context (built in FP64 from the lattice Green's function) against the oracle's
    column solves (Eq. action) for corner, edge and interior points of Omega_0, both components."""
    w, lev, sd = setup
    ctx = gpu_context(w, precision=1)
    n2 = 2 * sd.n_sd
    assert ctx.stats()["n_sd"] == sd.n_sd
    mid = (sd.nj // 2) * sd.ni + sd.ni // 2
    for col in (0, sd.ni - 1, mid, sd.n_sd - 1, sd.n_sd + mid, n2 - 1):
        ref = oib.b0_column(sd, col, w["re"], w["dt"])
        got = ctx.operator_entries(np.arange(n2), np.full(n2, col))
        assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref)), col
    ctx.close()


@pytest.mark.parametrize("precision,bound", [(0, 1e-10), (1, 2e-5)])
def test_no_slip_after_corrector_at_full_size(lib, setup, precision, bound):
    """After each step P E0 (C s + q_inf) equals the flag's node velocities T zeta_{n+1} (Eq. corrector2),
    with the CUDA graph the bench replays; FP32 fields bound the FP32 path's identity."""
    w, lev, sd = setup
    ctx = gpu_context(w, precision=precision)
    ctx.advance(6)
    u, v = og.faces_from_s(ctx.field(0, 1), lev)
    e0q = sd.e0(u + w["uinf"][0], v + w["uinf"][1])
    nb = w["bodies"][0]["n_pts"]
    idx, wts = ctx.interp(nb)
    ub = np.stack([(wts * e0q[idx]).sum(1), (wts * e0q[idx + sd.n_sd]).sum(1)], axis=1)
    _, zeta, _ = ctx.beam_state(0)
    vel = np.zeros((nb, 2))
    vel[1:] = zeta[:, :2]                                   # node 0 is the clamp
    scale = max(1.0, np.max(np.abs(ub)))
    assert np.max(np.abs(ub - vel)) < bound * scale
    ctx.close()
