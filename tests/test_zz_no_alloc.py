"""GPU test of the allocation-free level solve (fsi_op_level_solve_noalloc).

The entry point serves callers that cannot call cudaMalloc themselves -- code that runs under a framework
whose allocator owns all device memory, or a callback that must not allocate -- by keeping its transform
scratch in a fixed array inside the library.  Here it is called through the C ABI with device buffers the
test owns, twice in a row with different inputs, and its results are compared with the allocating entry
point fsi_op_level_solve within the tolerances of the other parity tests (1e-12 FP64, 2e-5 FP32 relative);
on the two smaller grids they are also compared with the FP64 oracle's dense sine-transform solves of the same
right-hand sides, so that the check does not rest on a second CUDA path alone.  The file name makes pytest
collect it last.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("prec,nx,ny", [(0, 128, 64), (1, 256, 128), (0, 512, 512), (1, 1024, 512)])
def test_noalloc_level_solve_matches_allocating_entry_point(prec, nx, ny):
    import torch

    import paper_2103_06415_gb300 as p
    from paper_2103_06415_gb300 import _lib
    from paper_2103_06415_gb300 import workloads as wl

    lib = _lib.load()
    h, re, dt = 1.0 / nx, 150.0, 0.003
    dtype = torch.float64 if prec == 0 else torch.float32
    tol = 1e-12 if prec == 0 else 2e-5
    stream = torch.cuda.current_stream()
    for call in range(2):
        rhs = wl.random_rhs(ny - 1, nx - 1, seed=1000 * call + nx + ny)
        w_ref, s_ref = p.level_solve(rhs, h, re, dt, precision=prec)   # allocating entry point
        rhs_d = torch.tensor(rhs, dtype=dtype, device="cuda")
        w_d = torch.full((ny + 1, nx + 1), 7.0, dtype=dtype, device="cuda")   # ring must stay untouched
        s_d = torch.full((ny + 1, nx + 1), -3.0, dtype=dtype, device="cuda")
        rc = lib.fsi_op_level_solve_noalloc(prec, nx, ny, h, re, dt, ctypes.c_void_p(rhs_d.data_ptr()),
                                            ctypes.c_void_p(w_d.data_ptr()), ctypes.c_void_p(s_d.data_ptr()),
                                            ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.fsi_last_error_message()
        torch.cuda.synchronize()
        w = w_d.cpu().double().numpy()
        s = s_d.cpu().double().numpy()
        assert _rel(w[1:-1, 1:-1], w_ref) < tol
        assert _rel(s[1:-1, 1:-1], s_ref) < tol
        if nx * ny <= 256 * 128:   # the oracle: A_w w = rhs, -lap_h s = w with zero boundary values (Eq. predictor2)
            from oracle import grid as og
            lev = og.Level(nx, ny, h, 0.0, 0.0)
            zero = np.zeros(lev.shape)
            w_or = og.solve_aw(rhs, zero, lev, re, dt)
            s_or = og.solve_lap(w_or, zero, lev)
            assert _rel(w[1:-1, 1:-1], w_or) < tol
            assert _rel(s[1:-1, 1:-1], s_or) < tol
        ring = np.ones(w.shape, bool)
        ring[1:-1, 1:-1] = False
        assert np.all(w[ring] == 7.0) and np.all(s[ring] == -3.0)
    # the promise itself: after the calls above (kernels loaded, scratch set up), further calls change the
    # device's free memory by nothing
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        rc = lib.fsi_op_level_solve_noalloc(prec, nx, ny, h, re, dt, ctypes.c_void_p(rhs_d.data_ptr()),
                                            ctypes.c_void_p(w_d.data_ptr()), ctypes.c_void_p(s_d.data_ptr()),
                                            ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_level_solve_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_2103_06415_gb300 import _lib

    lib = _lib.load()
    nx = ny = 1024                                  # FP64 needs ~25 MB of scratch, above the 8 MiB limit
    buf = torch.zeros((ny + 1, nx + 1), dtype=torch.float64, device="cuda")
    rc = lib.fsi_op_level_solve_noalloc(0, nx, ny, 1.0 / nx, 100.0, 0.01, ctypes.c_void_p(buf.data_ptr()),
                                        ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()), None)
    assert rc == 3
    assert b"limit" in lib.fsi_last_error_message()
