"""GB300 implementation of the sub-domain strongly coupled immersed-boundary FSI method
(Nair & Goza): Python binding of the C ABI in ``include/ibfsi.h``.

``Context`` wraps one run: grid levels, bodies, the sub-domain Omega_0, the offline stage
(``precompute``, Algorithm 1) and the online stage (``advance``, Algorithm 2).  Arrays cross the
boundary as float64 numpy arrays; all computation happens in ``libibfsi.so``.
"""

import ctypes

import numpy as np

from . import _lib
from ._lib import (COUPLING_SUBDOMAIN, COUPLING_TRUE_E, FSI_PREC_FP32, FSI_PREC_FP64, FSI_PREC_MIXED,  # noqa: F401
                   FsiError, check)

__all__ = ["Context", "B0Set", "level_solve", "beam_solve", "flapping_kinematics", "fma_rate", "FSI_PREC_FP64", "FSI_PREC_FP32", "FSI_PREC_MIXED", "FsiError",
           "COUPLING_SUBDOMAIN", "COUPLING_TRUE_E"]


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Context:
    """One FSI run on the current CUDA device.

    grid: nx, ny (2^k or 3 * 2^k cells), n_levels, x0, y0, h, re, dt, uinf=(U, V)
    precision: FSI_PREC_FP64, FSI_PREC_FP32 or FSI_PREC_MIXED (float-pair fields, float transforms of every
    level's increments); stream: a cudaStream_t handle (int) or None.
    dst_method: 0 FFT sine transforms, 1 tensor-core sine-matrix GEMMs (FP32), 2 autotune per pass.
    coupling: COUPLING_SUBDOMAIN (the method) or COUPLING_TRUE_E (the true-E comparator; krylov_tol and
    krylov_max_iters control its conjugate-gradient solve, 0 = library defaults).
    fsi_solver: 0 automatic, 1 float inverse in shared memory, 2 distributed block-Jacobi inverse (large nf).
    allocator: None (cudaMalloc), or a pair (alloc, free) of callables: alloc(nbytes) -> device pointer (int,
    256-byte aligned, 0 when it cannot) and free(ptr), through which every device buffer of the context goes
    (fsi_exec_desc.dev_alloc); they are kept alive with the context.
    """

    def __init__(self, nx, ny, n_levels, x0, y0, h, re, dt, uinf=(1.0, 0.0), precision=FSI_PREC_FP64,
                 stream=None, max_iters=50, tol=1e-7, history_cap=1 << 16, use_graph=True, b0_method=0,
                 dst_method=0, coupling=COUPLING_SUBDOMAIN, krylov_tol=0.0, krylov_max_iters=0, fsi_solver=0,
                 allocator=None):
        self._lib = _lib.load()
        g = _lib.GridDesc(nx, ny, n_levels, x0, y0, h, re, dt, (ctypes.c_double * 2)(*uinf))
        x = _lib.ExecDesc(precision, ctypes.c_void_p(stream) if stream else None, max_iters, tol, history_cap,
                          1 if use_graph else 0, b0_method, dst_method, coupling, krylov_tol, krylov_max_iters,
                          fsi_solver)
        self._alloc_fns = None
        if allocator is not None:
            alloc, free = allocator
            self._alloc_fns = (_lib.DEV_ALLOC_FN(lambda n, user: alloc(n) or None),
                               _lib.DEV_FREE_FN(lambda p, user: free(p)))
            x.dev_alloc, x.dev_free = self._alloc_fns
        h_ = ctypes.c_void_p()
        check(self._lib.fsi_create(ctypes.byref(g), ctypes.byref(x), ctypes.byref(h_)), "fsi_create")
        self._h = h_
        self.nx, self.ny, self.n_levels = nx, ny, n_levels
        self.n_bodies = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fsi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- setup -------------------------------------------------------------------------------

    def add_torsional(self, hinge, theta0, n_pts, ds, inertia, damping, stiffness, theta_init, phi_init=0.0,
                      driver=None, hinge_offset=0.0, mass=0.0, cg_offset=0.0):
        """Torsional plate (App. A).  driver: id of a driven plate carrying the hinge at hinge_offset along
        it (Eq. newtonseldg; mass and cg_offset enter the pseudo-force moment, inertia is about the hinge)."""
        b = _lib.BodyDesc(_lib.FSI_BODY_TORSIONAL, n_pts, ds, (ctypes.c_double * 2)(*hinge), theta0, theta_init,
                          phi_init, inertia, damping, stiffness, None, None)
        if driver is not None:
            b.driver = driver + 1
            b.hinge_offset, b.mass, b.cg_offset = hinge_offset, mass, cg_offset
        bid = ctypes.c_int()
        check(self._lib.fsi_add_body(self._h, ctypes.byref(b), ctypes.byref(bid)), "fsi_add_body")
        self.n_bodies += 1
        return bid.value

    def add_deformable(self, clamp, theta0, n_pts, ds, mass_per_length, bending_stiffness, stretching_stiffness,
                       tip_angle=0.0):
        """Clamped flag of ``n_pts - 1`` corotational beam elements (Eq. beam, App. A); starts at rest with
        tip slope ``tip_angle``.  Deflection outputs are the tip displacement and its rate."""
        b = _lib.BodyDesc(_lib.FSI_BODY_DEFORMABLE, n_pts, ds, (ctypes.c_double * 2)(*clamp), theta0, tip_angle,
                          0.0, 0.0, 0.0, 0.0, None, None, mass_per_length, bending_stiffness, stretching_stiffness)
        bid = ctypes.c_int()
        check(self._lib.fsi_add_body(self._h, ctypes.byref(b), ctypes.byref(bid)), "fsi_add_body")
        self.n_bodies += 1
        return bid.value

    def add_driven(self, ref, s_lo, n_pts, ds, a0, beta, sigma_t, sigma_r, freq=1.0):
        """Rigid plate with the prescribed heave and pitch of Sec. 5.1 (reference point ref, points at
        s_lo + j ds along (sin, -cos)(alpha1))."""
        b = _lib.BodyDesc(_lib.FSI_BODY_DRIVEN, n_pts, ds, (ctypes.c_double * 2)(*ref), 0, 0, 0, 0, 0, 0, None, None)
        b.kinematics = (ctypes.c_double * 5)(a0, beta, sigma_t, sigma_r, freq)
        b.s_lo = s_lo
        bid = ctypes.c_int()
        check(self._lib.fsi_add_body(self._h, ctypes.byref(b), ctypes.byref(bid)), "fsi_add_body")
        self.n_bodies += 1
        return bid.value

    def add_rigid(self, pts, ds, ur=None, append=False):
        """Rigid points with prescribed velocity ur (default 0).  append: the (fixed) points join Omega_0 and
        are interpolated with E itself (Sec. 3.1.1)."""
        pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
        urp = None
        if ur is not None:
            ur = np.ascontiguousarray(ur, dtype=np.float64).reshape(-1, 2)
            urp = _dp(ur)
        b = _lib.BodyDesc(_lib.FSI_BODY_RIGID, len(pts), ds, (ctypes.c_double * 2)(0, 0), 0, 0, 0, 0, 0, 0,
                          _dp(pts), urp)
        b.append_to_subdomain = 1 if append else 0
        bid = ctypes.c_int()
        check(self._lib.fsi_add_body(self._h, ctypes.byref(b), ctypes.byref(bid)), "fsi_add_body")
        self.n_bodies += 1
        return bid.value

    def set_subdomain(self, x_lo, x_hi, y_lo, y_hi):
        self.set_subdomain_boxes([(x_lo, x_hi, y_lo, y_hi)])

    def set_subdomain_boxes(self, boxes):
        """Omega_0 as the union of disjoint boxes (x_lo, x_hi, y_lo, y_hi), e.g. one per body (reading R16)."""
        arr = (_lib.Box * len(boxes))(*[_lib.Box(*b) for b in boxes])
        check(self._lib.fsi_set_subdomain(self._h, arr, len(boxes), None, 0), "fsi_set_subdomain")

    def precompute(self, drop_tol=0.0):
        check(self._lib.fsi_precompute(self._h, drop_tol), "fsi_precompute")

    def save_operator(self, path):
        """Write the precomputed operator (B0 or B0') to a file for runs with the same grid, Omega_0, Re, dt."""
        check(self._lib.fsi_save_operator(self._h, str(path).encode()), "fsi_save_operator")

    def save_state(self, path):
        """Checkpoint the run (everything the next step reads) to a file."""
        check(self._lib.fsi_save_state(self._h, str(path).encode()), "fsi_save_state")

    def load_state(self, path):
        """Resume from a checkpoint written by a context set up the same way (after precompute)."""
        check(self._lib.fsi_load_state(self._h, str(path).encode()), "fsi_load_state")

    def load_operator(self, path):
        """Offline stage from a file written by save_operator (in place of precompute)."""
        check(self._lib.fsi_load_operator(self._h, str(path).encode()), "fsi_load_operator")

    # -- online ------------------------------------------------------------------------------

    def advance(self, n_steps):
        check(self._lib.fsi_advance(self._h, n_steps), "fsi_advance")

    def sync(self):
        check(self._lib.fsi_sync(self._h), "fsi_sync")

    # -- outputs -----------------------------------------------------------------------------

    def forces(self, body=0):
        fx, fy, m = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(self._lib.fsi_get_forces(self._h, body, ctypes.byref(fx), ctypes.byref(fy), ctypes.byref(m)),
              "fsi_get_forces")
        return fx.value, fy.value, m.value

    def read_outputs_async(self, host_ptr, cap):
        """Enqueue a copy of every body's (fx, fy, moment, theta, phi) after the steps enqueued so far into the
        host memory at the integer address host_ptr (cap doubles, at least 5 per body; page-locked for the call
        not to wait); the values are there after the next sync."""
        check(self._lib.fsi_read_outputs_async(self._h, ctypes.c_void_p(host_ptr), int(cap)),
              "fsi_read_outputs_async")

    def deflection(self, body=0):
        th, ph = ctypes.c_double(), ctypes.c_double()
        check(self._lib.fsi_get_deflection(self._h, body, ctypes.byref(th), ctypes.byref(ph)), "fsi_get_deflection")
        return th.value, ph.value

    def history(self, body=0, cap=1 << 16):
        """Per-step array [n, 6]: fx, fy, moment, theta, phi, FSI iterations (oldest first)."""
        cols = []
        for field in range(6):
            out = np.zeros(cap)
            n = ctypes.c_int()
            check(self._lib.fsi_get_history(self._h, body, field, _dp(out), cap, ctypes.byref(n)), "fsi_get_history")
            cols.append(out[: n.value])
        return np.stack(cols, axis=1)

    def beam_state(self, body=0):
        """(chi, zeta, zetadot) of a flag: [n_pts - 1, 3] arrays of (x, y, theta) of nodes 1.. and rates."""
        n = ctypes.c_int()
        check(self._lib.fsi_get_beam_state(self._h, body, None, None, None, 0, ctypes.byref(n)), "fsi_get_beam_state")
        out = [np.zeros(n.value) for _ in range(3)]
        check(self._lib.fsi_get_beam_state(self._h, body, _dp(out[0]), _dp(out[1]), _dp(out[2]), n.value,
                                           ctypes.byref(n)), "fsi_get_beam_state")
        return tuple(o.reshape(-1, 3) for o in out)

    def field(self, level, which):
        out = np.zeros((self.ny + 1, self.nx + 1))
        check(self._lib.fsi_get_field(self._h, level, which, _dp(out)), "fsi_get_field")
        return out

    def set_field(self, level, which, arr):
        arr = np.ascontiguousarray(arr, dtype=np.float64)
        assert arr.shape == (self.ny + 1, self.nx + 1)
        check(self._lib.fsi_set_field(self._h, level, which, _dp(arr)), "fsi_set_field")

    def operator_entries(self, rows, cols):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        out = np.zeros(len(rows))
        check(self._lib.fsi_get_operator_entries(self._h, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                                 cols.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(rows),
                                                 _dp(out)), "fsi_get_operator_entries")
        return out

    def factor_operator(self, tau_rel=1e-10):
        """Cholesky factor of B0 + tau I on the device; returns (tau, seconds)."""
        tau, sec = ctypes.c_double(), ctypes.c_double()
        check(self._lib.fsi_factor_operator(self._h, tau_rel, ctypes.byref(tau), ctypes.byref(sec)),
              "fsi_factor_operator")
        return tau.value, sec.value

    def factor_entries(self, rows, cols):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        out = np.zeros(len(rows))
        check(self._lib.fsi_get_factor_entries(self._h, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                               cols.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(rows),
                                               _dp(out)), "fsi_get_factor_entries")
        return out

    def interp(self, n_points):
        idx = np.zeros(4 * n_points, dtype=np.int64)
        w = np.zeros(4 * n_points)
        check(self._lib.fsi_get_interp(self._h, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(w),
                                       n_points), "fsi_get_interp")
        return idx.reshape(-1, 4), w.reshape(-1, 4)

    KERNEL_CLASSES = {"xf": 1, "ysolve": 2, "xi": 3, "fsi": 4, "rhs": 5, "src": 6, "ring": 7}

    def profile_kernel(self, name, n_steps):
        """Run n_steps eager steps timing every launch of one kernel class; returns (mean ms, launches)."""
        ms, n = ctypes.c_double(), ctypes.c_int()
        check(self._lib.fsi_profile_kernel(self._h, self.KERNEL_CLASSES[name], n_steps, ctypes.byref(ms),
                                           ctypes.byref(n)), "fsi_profile_kernel")
        return ms.value, n.value

    PHASES = ("points_rhs", "assemble_PB0PT", "inverse_refresh", "inverse_rebuild", "refine_solves",
              "residuals", "dtheta", "outputs", "ns_xk_columns", "ns_new_x_rows", "ns_reload_x", "solve_d",
              "residual_rows_barrier", "residual_gather", "a_points_warps0_3", "a_flags_warps4_7",
              "a_wait_points", "a_point_tables", "a_owned_rows", "a_wait_flags", "a_flag_term", "a_grid_barrier",
              "a_rhs", "solve_d_rows_barrier")

    def set_phase_timing(self, on):
        """Phase timers of the FSI kernel on (counters cleared) or off (the default)."""
        check(self._lib.fsi_set_phase_timing(self._h, 1 if on else 0), "fsi_set_phase_timing")

    def phase_times(self):
        """Accumulated device wall time (ms) per phase of the FSI-iteration kernel."""
        out = np.zeros(len(self.PHASES))
        check(self._lib.fsi_get_phase_times(self._h, _dp(out), len(self.PHASES)), "fsi_get_phase_times")
        return dict(zip(self.PHASES, out.tolist()))

    def stats(self):
        s = _lib.Stats()
        check(self._lib.fsi_get_stats(self._h, ctypes.byref(s)), "fsi_get_stats")
        out = {k: getattr(s, k) for k, _ in s._fields_}
        out["dst_gemm"] = list(s.dst_gemm)
        out["dst_us"] = {"fft": list(s.dst_us)[:3], "gemm": list(s.dst_us)[3:]}
        return out

    def small_system(self):
        """K of the last FSI iteration (Eq. stress2), nf x nf, x-components of all points then y."""
        nf = self.stats()["nf"]
        out = np.zeros((nf, nf))
        n = ctypes.c_int()
        check(self._lib.fsi_get_small_system(self._h, _dp(out), nf * nf, ctypes.byref(n)), "fsi_get_small_system")
        return out


class B0Set:
    """B0 of several independent Omega_0 boxes on one grid, built together (``fsi_b0_set_build``).

    boxes: list of (x_lo, x_hi, y_lo, y_hi); method 0 = lattice Green's function, 1 = one DST solve per
    column (Algorithm 1) in the given precision."""

    def __init__(self, nx, ny, x0, y0, h, re, dt, boxes, method=0, precision=FSI_PREC_FP64, stream=None):
        self._lib = _lib.load()
        g = _lib.GridDesc(nx, ny, 1, x0, y0, h, re, dt, (ctypes.c_double * 2)(1.0, 0.0))
        x = _lib.ExecDesc(precision, ctypes.c_void_p(stream) if stream else None, 50, 1e-7, 16, 0, method)
        arr = (_lib.Box * len(boxes))(*[_lib.Box(*b) for b in boxes])
        h_ = ctypes.c_void_p()
        check(self._lib.fsi_b0_set_build(ctypes.byref(g), ctypes.byref(x), arr, len(boxes), ctypes.byref(h_)),
              "fsi_b0_set_build")
        self._h = h_
        self.n_boxes = len(boxes)

    def box(self, k):
        v = [ctypes.c_int() for _ in range(5)]
        check(self._lib.fsi_b0_set_box(self._h, k, *[ctypes.byref(a) for a in v]), "fsi_b0_set_box")
        i_lo, i_hi, j_lo, j_hi, n_sd = (a.value for a in v)
        return dict(i_lo=i_lo, i_hi=i_hi, j_lo=j_lo, j_hi=j_hi, n_sd=n_sd)

    def entries(self, k, rows, cols):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        out = np.zeros(len(rows))
        check(self._lib.fsi_b0_set_entries(self._h, k, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           cols.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(rows),
                                           _dp(out)), "fsi_b0_set_entries")
        return out

    def stats(self):
        sec, nbytes = ctypes.c_double(), ctypes.c_size_t()
        check(self._lib.fsi_b0_set_stats(self._h, ctypes.byref(sec), ctypes.byref(nbytes)), "fsi_b0_set_stats")
        return dict(seconds=sec.value, device_bytes=nbytes.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fsi_b0_set_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def level_solve(rhs, h, re, dt, precision=FSI_PREC_FP64, dst_method=0):
    """``w = A_w^{-1} rhs``, ``s = (-lap_h)^{-1} w`` on one level with zero boundary values (interior arrays).
    dst_method: 0 FFT passes, 1 tensor-core sine-matrix GEMMs (FP32), 2 autotuned per pass."""
    lib = _lib.load()
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    ny1, nx1 = rhs.shape
    w = np.zeros_like(rhs)
    s = np.zeros_like(rhs)
    check(lib.fsi_op_level_solve_ex(precision, dst_method, nx1 + 1, ny1 + 1, h, re, dt, _dp(rhs), _dp(w), _dp(s)),
          "fsi_op_level_solve_ex")
    return w, s


def flapping_kinematics(params, t):
    """(X1, X1', X1'', alpha1, alpha1', alpha1'') of a driven plate at time t as the library evaluates them
    (host computation; params = A0, beta, sigma_t, sigma_r, f)."""
    lib = _lib.load()
    p = np.ascontiguousarray(params, dtype=np.float64)
    out = np.zeros(6)
    check(lib.fsi_op_flapping_kinematics(_dp(p), float(t), _dp(out)), "fsi_op_flapping_kinematics")
    return out


def beam_solve(n_el, ds, mu, ei, ea, clamp, dt, chi, chi_n, zeta_n, zetadot_n, ref, b):
    """Structural linearisation of a flag on the GPU (see ``fsi_op_beam_solve``): returns (r_zeta, x) with
    r_zeta = M((4/dt^2)(chi_n - chi) + (4/dt) zeta_n + zetadot_n) - R(chi) and x = J_d(chi)^-1 b."""
    lib = _lib.load()
    arrs = [np.ascontiguousarray(v, dtype=np.float64).ravel() for v in (chi, chi_n, zeta_n, zetadot_n, ref, b)]
    nd = 3 * n_el
    assert all(v.size == nd for v in arrs)
    rz, x = np.zeros(nd), np.zeros(nd)
    check(lib.fsi_op_beam_solve(n_el, ds, mu, ei, ea, clamp[0], clamp[1], dt, *[_dp(v) for v in arrs], _dp(rz),
                                _dp(x)), "fsi_op_beam_solve")
    return rz, x


def fma_rate(precision):
    lib = _lib.load()
    r = ctypes.c_double()
    check(lib.fsi_op_fma_rate(precision, ctypes.byref(r)), "fsi_op_fma_rate")
    return r.value


class Server:
    """Continuous-batching server (include/ibfsi_server.h): runs are admitted as the HBM budget allows and
    advanced together, one step of every resident run per tick."""

    def __init__(self, hbm_budget_bytes, max_active=0):
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        check(self._lib.fsi_server_create(int(hbm_budget_bytes), max_active, ctypes.byref(h)), "fsi_server_create")
        self._h = h
        self._hist = {}   # run id -> history array the server fills at retirement (kept alive until polled)

    def submit(self, w, body, n_steps, precision=FSI_PREC_FP32, tag=0, history=False):
        """w: grid/sub-domain description (workloads dict keys); body: a torsional body dict (kind "torsional",
        the default) or a deformable one (kind "deformable": clamp, theta0, mass, ei, ea, tip_angle).  history:
        the poll result then carries the run's per-step history [n_steps, 6]."""
        g = _lib.GridDesc(w["nx"], w["ny"], w["n_levels"], w["x0"], w["y0"], w["h"], w["re"], w["dt"],
                          (ctypes.c_double * 2)(*w["uinf"]))
        if body.get("kind", "torsional") == "deformable":
            b = _lib.BodyDesc(_lib.FSI_BODY_DEFORMABLE, body["n_pts"], w["ds"], (ctypes.c_double * 2)(*body["clamp"]),
                              body["theta0"], body["tip_angle"], 0.0, 0.0, 0.0, 0.0, None, None, body["mass"],
                              body["ei"], body["ea"])
        else:
            b = _lib.BodyDesc(_lib.FSI_BODY_TORSIONAL, body["n_pts"], w["ds"], (ctypes.c_double * 2)(*body["hinge"]),
                              body["theta0"], body["theta"], 0.0, body["inertia"], body["damping"], body["stiffness"],
                              None, None)
        box = _lib.Box(*w["sd_box"])
        out = np.full((n_steps, 6), np.nan) if history else None
        req = _lib.Request(g, b, box, precision, n_steps, tag, _dp(out) if history else None)
        rid = ctypes.c_uint64()
        check(self._lib.fsi_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid)), "fsi_server_submit")
        if history:
            self._hist[rid.value] = out
        return rid.value

    def step(self):
        n = ctypes.c_int()
        check(self._lib.fsi_server_step(self._h, ctypes.byref(n)), "fsi_server_step")
        return n.value

    def poll(self, cap=256):
        buf = (_lib.Result * cap)()
        n = ctypes.c_int()
        check(self._lib.fsi_server_poll(self._h, buf, cap, ctypes.byref(n)), "fsi_server_poll")
        out = [{k: getattr(buf[i], k) for k, _ in _lib.Result._fields_} for i in range(n.value)]
        for r in out:
            hist = self._hist.pop(r["id"], None)
            if hist is not None:
                r["history"] = hist[: r["steps"]]
        return out

    def stats(self):
        s = _lib.ServerStats()
        check(self._lib.fsi_server_get_stats(self._h, ctypes.byref(s)), "fsi_server_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fsi_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
