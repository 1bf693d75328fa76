"""Several contexts of different sizes in one process (needs a GB300 and the library): kernels whose dynamic
shared memory depends on the run keep working for the larger run after a smaller one was set up."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("coupling", [0, 1])
def test_larger_context_runs_after_a_smaller_one_is_set_up(coupling):
    big = wl.small_flapping() if coupling == 1 else wl.small_flag()    # more shared memory per launch
    small = wl.small_plate()
    ref = gpu_context(big, coupling=coupling)
    ref.advance(6)
    h_ref = ref.history(len(big["bodies"]) - 1)
    ref.close()
    c_big = gpu_context(big, coupling=coupling)
    c_small = gpu_context(small, coupling=coupling)
    c_small.advance(2)
    c_big.advance(6)
    assert np.array_equal(c_big.history(len(big["bodies"]) - 1), h_ref)
    c_small.close()
    c_big.close()


def test_phase_timers_are_opt_in_and_leave_results_unchanged():
    """The FSI kernel's phase timers are off by default (no counts); turned on they count the steps that
    follow; the run's histories are the same bits with them on, off, and toggled mid-run (the captured step
    is captured anew)."""
    from paper_2103_06415_gb300 import workloads as wl
    from runners import gpu_context
    w = wl.small_flag()
    ref = gpu_context(w)
    ref.advance(9)
    want = ref.history(0)
    assert sum(ref.phase_times().values()) == 0.0
    ref.close()
    c = gpu_context(w)
    c.advance(3)
    c.set_phase_timing(True)
    c.advance(3)
    t = c.phase_times()
    assert t["points_rhs"] > 0 and t["outputs"] > 0
    c.set_phase_timing(False)
    c.advance(3)
    assert (c.history(0) == want).all()
    c.close()


def test_asynchronous_output_reads_match_the_synchronising_ones():
    """fsi_read_outputs_async enqueued after every step into page-locked memory gives, once the stream is
    synchronised, each step's forces and deflections of every body: equal to the step's history row (the
    synchronising reads) and to fsi_get_forces / fsi_get_deflection after the last step; too small a buffer
    is rejected."""
    import torch

    from paper_2103_06415_gb300 import _lib
    w = wl.small_mixed_bodies()       # two flags and a torsional plate
    nbody, n = len(w["bodies"]), 7
    c = gpu_context(w)
    out = torch.zeros((n, 5 * nbody), dtype=torch.float64, pin_memory=True)
    row = 5 * nbody * 8
    for k in range(n):
        c.advance(1)
        c.read_outputs_async(out.data_ptr() + k * row, 5 * nbody)
    c.sync()
    got = out.numpy()
    for b in range(nbody):
        h = c.history(b)[-n:]
        assert np.array_equal(got[:, 5 * b:5 * b + 5], h[:, :5]), b
        assert np.array_equal(got[-1, 5 * b:5 * b + 3], np.array(c.forces(b)))
        assert np.array_equal(got[-1, 5 * b + 3:5 * b + 5], np.array(c.deflection(b)))
    lib = _lib.load()
    assert lib.fsi_read_outputs_async(c._h, out.data_ptr(), 5 * nbody - 1) == 1   # FSI_ERR_INVALID_ARG
    c.close()
