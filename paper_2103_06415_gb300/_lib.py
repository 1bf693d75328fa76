"""ctypes binding of ``libibfsi.so`` (argument marshalling only; every step runs in the CUDA library).

The structures mirror ``include/ibfsi.h``.  Loading fails loudly if the library has not been built:
there is no fallback implementation.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libibfsi.so")

FSI_PREC_FP64 = 0
COUPLING_SUBDOMAIN = 0  # E0, P and the precomputed B0 (Sec. 3)
COUPLING_TRUE_E = 1     # E, E^T at the body points, Krylov solve per FSI iteration (Sec. 2.2)
FSI_PREC_FP32 = 1
FSI_PREC_MIXED = 2      # double level fields, float transforms, finest level in increment form
FSI_BODY_RIGID = 0
FSI_BODY_TORSIONAL = 1
FSI_BODY_DEFORMABLE = 2
FSI_BODY_DRIVEN = 3

STATUS = {
    0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "UNSUPPORTED", 4: "BODY_OUTSIDE_SUBDOMAIN",
    5: "NOT_CONVERGED", 6: "NONFINITE", 7: "TIMEOUT", 8: "CUDA", 9: "STATE",
}


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("h", ctypes.c_double),
                ("re", ctypes.c_double), ("dt", ctypes.c_double), ("uinf", ctypes.c_double * 2)]


DEV_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
DEV_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class ExecDesc(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("stream", ctypes.c_void_p), ("max_iters", ctypes.c_int),
                ("tol", ctypes.c_double), ("history_cap", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("b0_method", ctypes.c_int), ("dst_method", ctypes.c_int), ("coupling", ctypes.c_int),
                ("krylov_tol", ctypes.c_double), ("krylov_max_iters", ctypes.c_int), ("fsi_solver", ctypes.c_int),
                ("dev_alloc", DEV_ALLOC_FN), ("dev_free", DEV_FREE_FN), ("dev_alloc_user", ctypes.c_void_p)]


class BodyDesc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("n_pts", ctypes.c_int), ("ds", ctypes.c_double),
                ("hinge", ctypes.c_double * 2), ("theta0", ctypes.c_double), ("theta_init", ctypes.c_double),
                ("phi_init", ctypes.c_double), ("inertia", ctypes.c_double), ("damping", ctypes.c_double),
                ("stiffness", ctypes.c_double), ("pts", ctypes.POINTER(ctypes.c_double)),
                ("ur", ctypes.POINTER(ctypes.c_double)), ("mass_per_length", ctypes.c_double),
                ("bending_stiffness", ctypes.c_double), ("stretching_stiffness", ctypes.c_double),
                ("kinematics", ctypes.c_double * 5), ("s_lo", ctypes.c_double), ("driver", ctypes.c_int),
                ("hinge_offset", ctypes.c_double), ("mass", ctypes.c_double), ("cg_offset", ctypes.c_double),
                ("append_to_subdomain", ctypes.c_int)]


class Box(ctypes.Structure):
    _fields_ = [("x_lo", ctypes.c_double), ("x_hi", ctypes.c_double), ("y_lo", ctypes.c_double),
                ("y_hi", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("steps_done", ctypes.c_int64), ("last_iters", ctypes.c_int), ("max_iters_seen", ctypes.c_int),
                ("n_sd", ctypes.c_int), ("nf", ctypes.c_int), ("b0_seconds", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("launches_per_step", ctypes.c_int),
                ("last_solves", ctypes.c_int), ("inverse_rebuilds", ctypes.c_int),
                ("dst_gemm", ctypes.c_int * 3), ("dst_us", ctypes.c_double * 6), ("last_refreshes", ctypes.c_int),
                ("b0_nnz", ctypes.c_int64), ("b0_window", ctypes.c_int), ("last_krylov_iters", ctypes.c_int),
                ("krylov_iters_total", ctypes.c_int64)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_INT = ctypes.c_int

SIGNATURES = {
    "fsi_status_string": (ctypes.c_char_p, [_INT]),
    "fsi_last_error_message": (ctypes.c_char_p, []),
    "fsi_create": (_INT, [ctypes.POINTER(GridDesc), ctypes.POINTER(ExecDesc), ctypes.POINTER(_P)]),
    "fsi_add_body": (_INT, [_P, ctypes.POINTER(BodyDesc), ctypes.POINTER(_INT)]),
    "fsi_set_subdomain": (_INT, [_P, ctypes.POINTER(Box), _INT, _D, _INT]),
    "fsi_precompute": (_INT, [_P, ctypes.c_double]),
    "fsi_advance": (_INT, [_P, _INT]),
    "fsi_sync": (_INT, [_P]),
    "fsi_get_forces": (_INT, [_P, _INT, _D, _D, _D]),
    "fsi_get_deflection": (_INT, [_P, _INT, _D, _D]),
    "fsi_read_outputs_async": (_INT, [_P, _P, _INT]),
    "fsi_get_history": (_INT, [_P, _INT, _INT, _D, _INT, ctypes.POINTER(_INT)]),
    "fsi_get_beam_state": (_INT, [_P, _INT, _D, _D, _D, _INT, ctypes.POINTER(_INT)]),
    "fsi_get_field": (_INT, [_P, _INT, _INT, _D]),
    "fsi_set_field": (_INT, [_P, _INT, _INT, _D]),
    "fsi_get_operator_entries": (_INT, [_P, _I64, _I64, _INT, _D]),
    "fsi_get_interp": (_INT, [_P, _I64, _D, _INT]),
    "fsi_factor_operator": (_INT, [_P, ctypes.c_double, _D, _D]),
    "fsi_get_factor_entries": (_INT, [_P, _I64, _I64, _INT, _D]),
    "fsi_get_stats": (_INT, [_P, ctypes.POINTER(Stats)]),
    "fsi_get_small_system": (_INT, [_P, _D, ctypes.c_int64, ctypes.POINTER(_INT)]),
    "fsi_debug_set_wait_limit": (_INT, [_P, ctypes.c_uint, _INT]),
    "fsi_profile_kernel": (_INT, [_P, _INT, _INT, _D, ctypes.POINTER(_INT)]),
    "fsi_get_phase_times": (_INT, [_P, _D, _INT]),
    "fsi_set_phase_timing": (_INT, [_P, _INT]),
    "fsi_destroy": (None, [_P]),
    "fsi_op_level_solve": (_INT, [_INT, _INT, _INT, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D, _D]),
    "fsi_op_level_solve_ex": (_INT, [_INT, _INT, _INT, _INT, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D,
                                     _D, _D]),
    "fsi_op_fma_rate": (_INT, [_INT, _D]),
    "fsi_op_flapping_kinematics": (_INT, [_D, ctypes.c_double, _D]),
    "fsi_save_operator": (_INT, [_P, ctypes.c_char_p]),
    "fsi_load_operator": (_INT, [_P, ctypes.c_char_p]),
    "fsi_save_state": (_INT, [_P, ctypes.c_char_p]),
    "fsi_load_state": (_INT, [_P, ctypes.c_char_p]),
    "fsi_op_beam_solve": (_INT, [_INT] + [ctypes.c_double] * 7 + [_D] * 8),
    "fsi_op_level_solve_noalloc": (_INT, [_INT, _INT, _INT, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         _P, _P, _P, _P]),
}

_lib = None


def load():
    """Load ``libibfsi.so`` (raises if it is missing: build it with ``paper_2103_06415_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libibfsi.so is not built; run `python -m paper_2103_06415_gb300.build` "
                          "(the CUDA library is the only implementation)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FsiError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = "%s: %s" % (where, STATUS.get(code, code))
        if code == 8 and _lib is not None:
            msg += " (%s)" % _lib.fsi_last_error_message().decode()
        super().__init__(msg)


def check(code, where):
    if code != 0:
        raise FsiError(code, where)
    return code


class Request(ctypes.Structure):
    _fields_ = [("grid", GridDesc), ("body", BodyDesc), ("box", Box), ("precision", ctypes.c_int),
                ("n_steps", ctypes.c_int), ("tag", ctypes.c_uint64), ("history_out", ctypes.POINTER(ctypes.c_double))]


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int), ("steps", ctypes.c_int),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("moment", ctypes.c_double),
                ("theta", ctypes.c_double), ("phi", ctypes.c_double), ("mean_step_ms", ctypes.c_double),
                ("p50_step_ms", ctypes.c_double), ("p99_step_ms", ctypes.c_double), ("wait_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int), ("active", ctypes.c_int), ("finished", ctypes.c_int),
                ("admitting", ctypes.c_int), ("bytes_in_use", ctypes.c_size_t), ("ticks", ctypes.c_longlong), ("run_steps", ctypes.c_longlong),
                ("cell_steps", ctypes.c_double), ("busy_ms", ctypes.c_double)]


SIGNATURES.update({
    "fsi_server_create": (_INT, [ctypes.c_size_t, _INT, ctypes.POINTER(_P)]),
    "fsi_server_submit": (_INT, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "fsi_server_step": (_INT, [_P, ctypes.POINTER(_INT)]),
    "fsi_server_poll": (_INT, [_P, ctypes.POINTER(Result), _INT, ctypes.POINTER(_INT)]),
    "fsi_server_get_stats": (_INT, [_P, ctypes.POINTER(ServerStats)]),
    "fsi_server_destroy": (None, [_P]),
})

SIGNATURES.update({
    "fsi_b0_set_build": (_INT, [ctypes.POINTER(GridDesc), ctypes.POINTER(ExecDesc), ctypes.POINTER(Box), _INT,
                                ctypes.POINTER(_P)]),
    "fsi_b0_set_box": (_INT, [_P, _INT, ctypes.POINTER(_INT), ctypes.POINTER(_INT), ctypes.POINTER(_INT),
                              ctypes.POINTER(_INT), ctypes.POINTER(_INT)]),
    "fsi_b0_set_entries": (_INT, [_P, _INT, _I64, _I64, _INT, _D]),
    "fsi_b0_set_stats": (_INT, [_P, _D, ctypes.POINTER(ctypes.c_size_t)]),
    "fsi_b0_set_destroy": (None, [_P]),
})
