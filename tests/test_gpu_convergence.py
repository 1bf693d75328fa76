"""Physics sanity (not parity): the observed spatial order of the torsional-plate deflection under grid
refinement lies between first and second order, as for the paper's Richardson estimate p = 1.34 (Sec. 5.1;
immersed-boundary methods converge at first to second order).  Needs a GB300 and the library."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context

pytestmark = pytest.mark.gpu


def test_plate_deflection_converges_between_first_and_second_order():
    """plate_128's plate on 64^2, 128^2, 256^2 cells of the same domain, dt and ds refined with h, up to
    t = 1; p = log2(|theta_4h - theta_2h| / |theta_2h - theta_h|) on the coarse grid's time levels."""
    hist = {}
    for n in (64, 128, 256):
        w = wl.plate_128()
        h = 4.0 / n
        w.update(nx=n, ny=n, h=h, dt=0.002 * 128 / n, ds=h)
        w["bodies"][0]["n_pts"] = int(round(1.0 / h)) + 1
        ctx = gpu_context(w)
        ctx.advance(int(round(1.0 / w["dt"])))
        every = n // 64
        hist[n] = ctx.history(0)[every - 1::every, 3]
        ctx.close()
    m = min(len(v) for v in hist.values())
    a, b, c = hist[64][:m], hist[128][:m], hist[256][:m]
    p = np.log2(np.linalg.norm(a - b) / np.linalg.norm(b - c))
    assert 1.0 < p < 2.3, p
