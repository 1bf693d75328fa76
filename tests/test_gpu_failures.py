"""Failure detection without a GPU fault (needs a GB300 and the library): errors are latched status codes that
the host reads at the next synchronising call; the kernels never trap, so the CUDA context stays usable."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


def _status(lib, ctx):
    return ctx._lib.fsi_sync(ctx._h)


@pytest.mark.parametrize("coupling", [0, 1])
def test_iteration_limit_latches_not_converged(lib, coupling):
    """max_iters = 1 at a tolerance no single iteration meets: NOT_CONVERGED, outputs still readable."""
    w = wl.small_plate()
    ctx = gpu_context(w, max_iters=1, tol=1e-15, coupling=coupling)
    ctx.advance(3)
    assert _status(lib, ctx) == 5                          # FSI_ERR_NOT_CONVERGED
    import ctypes                                          # the C call fills its outputs with this status
    fx, fy, m = ctypes.c_double(np.nan), ctypes.c_double(np.nan), ctypes.c_double(np.nan)
    assert ctx._lib.fsi_get_forces(ctx._h, 0, ctypes.byref(fx), ctypes.byref(fy), ctypes.byref(m)) == 5
    assert np.isfinite(fx.value) and np.isfinite(fy.value)
    with pytest.raises(lib.FsiError):                      # the binding reports it as an error
        ctx.forces(0)
    ctx.close()


def test_injected_nan_latches_nonfinite(lib):
    w = wl.small_plate()
    ctx = gpu_context(w)
    ctx.advance(2)
    f = ctx.field(0, 0)
    f[10, 20] = np.nan                                     # a NaN in a host-supplied vorticity field
    ctx.set_field(0, 0, f)
    ctx.advance(2)
    assert _status(lib, ctx) == 6                          # FSI_ERR_NONFINITE
    ctx.close()


def test_body_leaving_omega0_latches_outside(lib):
    w = wl.small_plate()
    w["sd_box"] = (-0.2, 0.45, -0.3, 0.3)                  # does not hold the 0.5-long plate at 20 degrees
    ctx = gpu_context(w)
    ctx.advance(1)
    assert _status(lib, ctx) == 4                          # FSI_ERR_BODY_OUTSIDE_SUBDOMAIN
    ctx.close()


def test_first_error_wins_and_context_stays_usable(lib):
    w = wl.small_plate()
    bad = gpu_context(w, max_iters=1, tol=1e-15)
    bad.advance(2)
    f = bad.field(0, 0)
    f[5, 5] = np.inf
    bad.set_field(0, 0, f)
    bad.advance(2)
    assert _status(lib, bad) == 5                          # the first latched code is kept
    bad.close()
    good = gpu_context(w)                                  # the device is still healthy
    good.advance(5)
    assert _status(lib, good) == 0
    good.close()


def test_bounded_cross_cta_wait_latches_timeout(lib):
    """The FSI kernel's cross-CTA wait (warps 0-3 of every CTA, with a flag) polls a global arrival counter a
    bounded number of times.  Require one arrival that never comes and a short bound: every such wait runs
    out (no copies are in flight there), TIMEOUT is latched and read by the host, and the device stays
    healthy -- a new context on it reproduces an undisturbed run bit for bit."""
    w = wl.small_flag()
    ref = gpu_context(w)
    ref.advance(4)
    ref_hist = ref.history(0)
    ref.close()
    bad = gpu_context(w)
    bad.advance(2)
    assert _status(lib, bad) == 0
    assert bad._lib.fsi_debug_set_wait_limit(bad._h, 1 << 12, 1) == 0
    bad.advance(1)
    assert _status(lib, bad) == 7                          # FSI_ERR_TIMEOUT
    assert bad._lib.fsi_debug_set_wait_limit(bad._h, 0, 0) == 0
    bad.advance(1)
    assert _status(lib, bad) == 7                          # the first latched code is kept
    bad.close()
    good = gpu_context(w)
    good.advance(4)
    assert _status(lib, good) == 0
    assert np.array_equal(good.history(0), ref_hist)
    good.close()
