"""Checkpoint and resume (needs a GB300 and the library): n steps, save, load into a context set up the same
way, n steps equal 2n uninterrupted steps bit for bit."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


CASES = [("plate", dict(), 0), ("flag", dict(), 0), ("flapping", dict(), 0), ("plate_fp32", dict(precision=1), 0),
         ("plate_true_e", dict(coupling=1), 0), ("flag_eager", dict(use_graph=False), 0)]


def _workload(name):
    if name.startswith("plate"):
        return wl.small_plate()
    if name.startswith("flag"):
        return wl.small_flag()
    return wl.small_flapping()


@pytest.mark.parametrize("name,kw,_", CASES)
def test_resume_equals_uninterrupted_run(lib, tmp_path, name, kw, _):
    w = _workload(name)
    n = 7
    ref = gpu_context(w, **kw)
    ref.advance(2 * n)
    a = gpu_context(w, **kw)
    a.advance(n)
    path = tmp_path / "state.bin"
    a.save_state(path)
    a.close()
    b = gpu_context(w, **kw)
    b.load_state(path)
    b.advance(n)
    for body in range(len(w["bodies"])):
        assert np.array_equal(b.history(body), ref.history(body)), body
    for which in (0, 1):
        assert np.array_equal(b.field(0, which), ref.field(0, which))
    if w["bodies"][-1]["kind"] == "deformable":
        for x, y in zip(b.beam_state(0), ref.beam_state(0)):
            assert np.array_equal(x, y)
    assert b.stats()["steps_done"] == 2 * n


def test_state_file_errors(lib, tmp_path):
    w = wl.small_plate()
    a = gpu_context(w)
    a.advance(3)
    path = tmp_path / "state.bin"
    a.save_state(path)
    other = gpu_context(wl.small_flag())                  # another shape
    with pytest.raises(lib.FsiError):
        other.load_state(path)
    data = path.read_bytes()
    (tmp_path / "short.bin").write_bytes(data[: len(data) - 100])
    b = gpu_context(w)
    b.advance(2)
    before = b.history(0)
    with pytest.raises(lib.FsiError):
        b.load_state(tmp_path / "short.bin")
    assert np.array_equal(b.history(0), before)            # left unchanged
    with pytest.raises(lib.FsiError):
        b.load_state(tmp_path / "missing.bin")
