"""Saving and reusing the precomputed operator (needs a GB300 and the library): B0 depends only on the grid,
Omega_0, Re and dt, so a run that loads it takes exactly the steps of a run that built it (the reuse noted
after Algorithm 1), also with other body parameters."""

import numpy as np
import pytest

from paper_2103_06415_gb300 import workloads as wl

from runners import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2103_06415_gb300 as p
    return p


@pytest.mark.parametrize("drop_tol", [0.0, 0.007])
def test_loaded_operator_reproduces_the_built_one(lib, tmp_path, drop_tol):
    w = wl.small_plate()
    path = tmp_path / "b0.bin"
    a = gpu_context(w, drop_tol=drop_tol)
    a.save_operator(path)
    b = gpu_context(w, precompute=False)
    b.load_operator(path)
    sa, sb = a.stats(), b.stats()
    assert sa["b0_nnz"] == sb["b0_nnz"] and sa["b0_window"] == sb["b0_window"]
    rows = np.arange(0, 2 * sa["n_sd"], 37)
    cols = (rows * 7) % (2 * sa["n_sd"])
    assert np.array_equal(a.operator_entries(rows, cols), b.operator_entries(rows, cols))
    a.advance(10)
    b.advance(10)
    assert np.array_equal(a.history(0), b.history(0))
    a.close()
    b.close()


def test_operator_reused_for_other_body_parameters(lib, tmp_path):
    """A parametric study: the operator built for one spring stiffness serves another."""
    w = wl.small_plate()
    path = tmp_path / "b0.bin"
    gpu_context(w).save_operator(path)
    w2 = wl.small_plate()
    w2["bodies"][0]["stiffness"] = 2.0
    fresh = gpu_context(w2)
    reused = gpu_context(w2, precompute=False)
    reused.load_operator(path)
    fresh.advance(8)
    reused.advance(8)
    assert np.array_equal(fresh.history(0), reused.history(0))


def test_operator_file_errors(lib, tmp_path):
    w = wl.small_plate()
    path = tmp_path / "b0.bin"
    a = gpu_context(w)
    a.save_operator(path)
    w_re = wl.small_plate()
    w_re["re"] = 150.0                                   # another Reynolds number: another operator
    c = gpu_context(w_re, precompute=False)
    with pytest.raises(lib.FsiError):
        c.load_operator(path)
    c = gpu_context(w, precompute=False)
    with pytest.raises(lib.FsiError):
        c.load_operator(tmp_path / "missing.bin")
    data = path.read_bytes()
    (tmp_path / "short.bin").write_bytes(data[: len(data) // 2])
    c = gpu_context(w, precompute=False)
    with pytest.raises(lib.FsiError):
        c.load_operator(tmp_path / "short.bin")
    c = gpu_context(w, precompute=False)
    with pytest.raises(lib.FsiError):                   # nothing to save before the offline stage
        c.save_operator(tmp_path / "x.bin")
    t = gpu_context(w, coupling=1)
    with pytest.raises(lib.FsiError):                   # the true-E comparator has no operator
        t.save_operator(tmp_path / "x.bin")
