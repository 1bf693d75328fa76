"""CPU checks of the C-ABI library: it builds, loads, and exports every symbol the headers declare."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"\b(fsi_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_builds_and_exports_all_declared_symbols():
    from paper_2103_06415_gb300 import build as b
    lib = b.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (fsi_[a-z0-9_]+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= exported, sorted(declared - exported)


def test_binding_signatures_cover_headers_and_load():
    from paper_2103_06415_gb300 import _lib
    lib = _lib.load()
    assert set(_lib.SIGNATURES) == _declared()
    assert lib.fsi_status_string(4) == b"body point outside the sub-domain"


def test_invalid_arguments_are_rejected_without_a_gpu():
    from paper_2103_06415_gb300 import _lib
    import ctypes
    lib = _lib.load()
    g = _lib.GridDesc(100, 64, 1, 0, 0, 0.1, 100, 0.01, (ctypes.c_double * 2)(1, 0))   # nx not a power of two
    h = ctypes.c_void_p()
    assert lib.fsi_create(ctypes.byref(g), None, ctypes.byref(h)) == 1
    assert lib.fsi_advance(None, 1) == 1


def test_b0_set_arguments_are_rejected_without_a_gpu():
    from paper_2103_06415_gb300 import _lib
    import ctypes
    lib = _lib.load()
    g = _lib.GridDesc(64, 64, 1, -2.0, -2.0, 1.0 / 16, 100.0, 0.004, (ctypes.c_double * 2)(1, 0))
    x = _lib.ExecDesc(0, None, 50, 1e-7, 16, 0, 0)
    good = (_lib.Box * 1)(_lib.Box(-1.0, 1.0, -1.0, 1.0))
    empty = (_lib.Box * 1)(_lib.Box(5.0, 6.0, 5.0, 6.0))          # outside the grid after clipping
    h = ctypes.c_void_p()
    assert lib.fsi_b0_set_build(ctypes.byref(g), ctypes.byref(x), good, 0, ctypes.byref(h)) == 1
    assert lib.fsi_b0_set_build(None, ctypes.byref(x), good, 1, ctypes.byref(h)) == 1
    assert lib.fsi_b0_set_build(ctypes.byref(g), ctypes.byref(x), empty, 1, ctypes.byref(h)) == 1
    x.b0_method = 7
    assert lib.fsi_b0_set_build(ctypes.byref(g), ctypes.byref(x), good, 1, ctypes.byref(h)) == 1
    assert not h.value
    assert lib.fsi_b0_set_box(None, 0, None, None, None, None, None) == 1


def test_server_request_validation_without_a_gpu():
    import paper_2103_06415_gb300 as p
    from paper_2103_06415_gb300 import workloads as wl
    srv = p.Server(2 << 30)
    w = wl.serving_grid(128)
    body = dict(hinge=(0.0, 0.0), theta0=0.0, n_pts=33, inertia=1.0, damping=0.0, stiffness=0.5, theta=0.3)
    assert srv.submit(w, body, 10) == 1
    with pytest.raises(p.FsiError):                       # a request that can never fit the budget
        p.Server(1 << 20).submit(w, body, 10)
    st = srv.stats()
    assert st["queued"] == 1 and st["active"] == 0
    srv.close()
