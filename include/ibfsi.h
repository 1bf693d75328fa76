/*
 * ibfsi.h -- C ABI of the GB300 library for the sub-domain strongly coupled
 * immersed-boundary fluid-structure interaction method of Nair & Goza
 * ("A strongly coupled immersed boundary method for fluid-structure interaction
 * that mimics the efficiency of stationary body methods").
 *
 * The calls follow the paper's statement of the problem: a fluid grid of nested
 * levels (Sec. 5, multidomain far field), bodies (Sec. 2.1, Eqs. newtons-bct),
 * a fixed sub-domain Omega_0 (Sec. 3.1.1), the offline stage that precomputes
 * B0 = E0 C (C^T A C)^{-1} C^T E0^T (Algorithm 1, Eq. action) and the online
 * stage that advances the coupled system (Algorithm 2, Eqs. predictor2-corrector2).
 *
 * Conventions
 *  - Every call returns an fsi_status; no call aborts the process and device
 *    code never traps.  Errors detected on the device are latched in a status
 *    word and returned by the next synchronising call.
 *  - All pointers in this header are HOST pointers unless stated otherwise.
 *    Inputs are copied during the call; the caller keeps ownership of every
 *    buffer it passes and of every output buffer it provides.
 *  - The library owns its device memory (cudaMalloc); fsi_destroy frees it.
 *  - Work is issued on the stream given at creation (a cudaStream_t passed as
 *    void*; NULL = legacy default stream).  fsi_advance is asynchronous; the
 *    fsi_get_* calls synchronise that stream.
 *  - Floating-point inputs are double precision whatever the compute precision.
 */
#ifndef IBFSI_H
#define IBFSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FSI_OK = 0,
  FSI_ERR_INVALID_ARG = 1,
  FSI_ERR_OOM = 2,
  FSI_ERR_UNSUPPORTED = 3,
  FSI_ERR_BODY_OUTSIDE_SUBDOMAIN = 4, /* a body point left Omega_0 (Sec. 3.1.1 requires it to stay inside) */
  FSI_ERR_NOT_CONVERGED = 5,          /* FSI iteration exceeded max_iters (Algorithm 2 while-loop) */
  FSI_ERR_NONFINITE = 6,              /* NaN/Inf in the small system or in the forces */
  FSI_ERR_TIMEOUT = 7,
  FSI_ERR_CUDA = 8,                   /* a CUDA runtime call failed; see fsi_last_error_message */
  FSI_ERR_STATE = 9                   /* call made in the wrong stage (e.g. advance before precompute) */
} fsi_status;

typedef enum {
  FSI_PREC_FP64 = 0, /* every fluid transform and stencil in double */
  FSI_PREC_FP32 = 1, /* fluid transforms and stencils in float; B0, the small system, Newton update and
                        force reductions stay in double */
  FSI_PREC_MIXED = 2 /* as FSI_PREC_FP32, but the vorticity and streamfunction fields are kept in double and,
                        after the first step, the finest level is advanced in increment form: its float
                        transforms compute w^{n+1} - w^n and s^{n+1} - s^n, which are added to the double
                        fields (coarser levels: full float solves).  No tensor-core transforms
                        (dst_method 1: FSI_ERR_UNSUPPORTED; 2 keeps the FFT) and no coupling 1. */
} fsi_precision;

typedef enum { FSI_BODY_RIGID = 0, FSI_BODY_TORSIONAL = 1, FSI_BODY_DEFORMABLE = 2, FSI_BODY_DRIVEN = 3 } fsi_body_type;

/* Fluid grid (Sec. 2.2; multidomain of Sec. 5).  Level 0 is the finest: nx x ny cells of spacing h with
 * lower-left corner (x0, y0).  Level g has the same cell counts, spacing 2^g h and the same centre.
 * nx and ny must be 2^k or 3 * 2^k in [16, 2048] (the DST lengths N+1 = nx, ny; the sine transforms use
 * radix-4/2 stages and, for 3 * 2^k, one radix-3 stage); when one axis has 3 * 2^k cells, an axis of 2^k
 * cells may have at most 512 (e.g. 1536 x 768, 1536 x 512, 768 x 512); otherwise FSI_ERR_INVALID_ARG.
 * n_levels >= 1.
 * re = Reynolds number, dt = time step, uinf = free-stream velocity. */
typedef struct {
  int nx, ny, n_levels;
  double x0, y0, h;
  double re, dt;
  double uinf[2];
} fsi_grid_desc;

/* Execution options.  stream: cudaStream_t (NULL = default stream).  max_iters (<= 0 -> 50) and tol
 * (<= 0 -> 1e-7) control the FSI iteration of Algorithm 2 (convergence on max |dtheta|, Sec. 5).
 * history_cap: number of steps kept in the per-step output ring (<= 0 -> 1<<16).
 * use_graph: nonzero captures one time step into a CUDA graph and replays it. */
typedef struct {
  int precision;
  void* stream;
  int max_iters;
  double tol;
  int history_cap;
  int use_graph;
  int b0_method; /* 0: B0 from the lattice Green's function of (C^T A C)^{-1} (all columns at once, double);
                    1: one DST solve per column as in Algorithm 1, in the context's precision. Same matrix. */
  int dst_method; /* sine transforms of the fluid solves (Sec. 3.2.1): 0 FFT passes; 1 dense sine-matrix GEMMs
                     on the tensor cores (compensated 3xTF32, FP32 precision only, nx in [128, 1024], ny in [128, 512],
                     otherwise FSI_ERR_UNSUPPORTED); 2 autotune: time both for each of the three passes at
                     fsi_create and keep the faster (decisions are cached per grid shape for the process, so
                     equal grids take equal paths); FP64 contexts and unsupported sizes then use FFT. */
  int coupling; /* 0: the sub-domain method (E0, P and the precomputed B0 of Sec. 3).  1: the true E and E^T
                   at the body points (Sec. 2.2), the comparator of Sec. 5.1: each FSI iteration solves the
                   small system matrix-free by conjugate gradients with one finest-level (C^T A C)^-1 per
                   Krylov iteration (homogeneous boundary values); fsi_precompute then builds no B0, the
                   sub-domain box only bounds the body points (outside: FSI_ERR_BODY_OUTSIDE_SUBDOMAIN), and
                   only TORSIONAL and RIGID bodies (at most 1024 points) are supported (else
                   FSI_ERR_UNSUPPORTED at fsi_precompute).  With use_graph the FSI and Krylov loops run as
                   device-side graph loops (no host round trip per iteration). */
  double krylov_tol; /* coupling 1: stop when |r| <= krylov_tol |rhs| (<= 0 -> 1e-10 FP64, 1e-5 FP32) */
  int krylov_max_iters; /* coupling 1: Krylov iterations per FSI iteration (<= 0 -> 2 nf + 20); reaching it
                           without convergence latches FSI_ERR_NOT_CONVERGED */
  int fsi_solver; /* solver of the small system of Eq. stress2 (coupling 0): 0 automatic; 1 a float inverse of
                     K held in the shared memory of every CTA of the FSI kernel, refined in double (nf up to
                     about 230); 2 distributed: a block-Jacobi float inverse (one block per body, the body's
                     x and y rows) and K in global memory, up to 12 rows per CTA, refined in double against
                     the full K (nf up to 12 x the SM count; it converges when the bodies' cross coupling in
                     K is weak, exactly block-diagonal K for bodies farther apart than the window of B0').
                     0 takes 1 when it fits, else 2.  A size the choice cannot hold: FSI_ERR_UNSUPPORTED at
                     fsi_precompute; other values: FSI_ERR_INVALID_ARG. */
  /* Device memory through the caller's allocator (not part of the paper's method: the boundary's hook for a
   * host framework that owns device memory).  When dev_alloc is not NULL, every device buffer the context
   * (or the box set of fsi_b0_set_build) allocates -- the level fields and scratch, B0 or B0', the FSI
   * workspace, and the temporaries of the offline stage -- comes from dev_alloc(bytes, dev_alloc_user), which
   * returns device memory usable on the context's stream, aligned to 256 bytes, or NULL when it cannot
   * (the call then fails with FSI_ERR_OOM; a misaligned pointer is handed back to dev_free and treated the
   * same way).  Each such pointer is returned once through dev_free(ptr, dev_alloc_user): temporaries when
   * their stage ends, the rest at fsi_destroy.  The library never calls them concurrently from several host
   * threads for one context.  dev_alloc NULL: cudaMalloc and cudaFree (dev_free and dev_alloc_user ignored);
   * dev_alloc without dev_free: FSI_ERR_INVALID_ARG. */
  void* (*dev_alloc)(size_t bytes, void* user);
  void (*dev_free)(void* ptr, void* user);
  void* dev_alloc_user;
} fsi_exec_desc;

/* A body (Sec. 2.1).  TORSIONAL: a straight plate of n_pts points j = 0..n_pts-1 at
 * hinge + j*ds*(cos(theta0+theta), sin(theta0+theta)), rotating about the hinge on a spring
 * (inertia, damping, stiffness; Eq. newtons with g_t = 0); theta_init, phi_init = initial deflection and
 * angular velocity.  RIGID: n_pts fixed points pts[2*j], pts[2*j+1] with prescribed velocity ur (same
 * layout; NULL = stationary).
 * DEFORMABLE (Eq. beam, App. A): a flag clamped at hinge, undeformed along the angle theta0, discretised as
 * n_pts - 1 two-dimensional corotational Euler-Bernoulli beam elements of length ds whose nodes are the
 * body points (node 0 is the clamp).  Material per unit length: mass_per_length (mass ratio, > 0),
 * bending_stiffness EI (> 0), stretching_stiffness EA (> 0).  Lumped mass (mass_per_length*ds per free node,
 * half at the tip; rotary inertia mass*ds^2/12), trapezoidal Newmark in time, J_d = 4M/dt^2 + K(chi) at the
 * iterate (Eqs. stress2, dchi2).  theta_init = initial tip slope: the flag starts at rest in the
 * inextensible shape with slope angle theta_init*(2 s/L - s^2/L^2) along its length L; phi_init must be 0.
 * For this type fsi_get_deflection and history fields 3, 4 report the tip displacement normal to the
 * undeformed flag and its rate.  n_pts >= 2.
 * DRIVEN (Sec. 5.1): a rigid plate with prescribed heave and pitch.  hinge = its reference point (the pitch
 * axis); at time t it is displaced by (X1(t), 0) and the plate lies along (sin, -cos)(alpha1(t)) (straight
 * down at alpha1 = 0), points j = 0..n_pts-1 at s_lo + j*ds along it.  kinematics = {A0, beta, sigma_t,
 * sigma_r, f}: X1 = (A0/2) G_t(f t)/max G_t C(f t), alpha1 = -beta G_r(f t)/max G_r with
 * G_t(tau) = int_0^tau tanh(sigma_t cos(2 pi u)) du, G_r = tanh(sigma_r cos(2 pi tau)),
 * C(tau) = (tanh(8 tau - 2) + tanh 2)/(1 + tanh 2).  A0 >= 0, beta finite, sigma_t, sigma_r, f > 0.
 * A TORSIONAL body with driver = k > 0 is hinged on the DRIVEN body with id k - 1 (added before it), at
 * hinge_offset (L1) along that plate from its reference point; its points lie along the driven plate's
 * direction turned by theta (theta0 must be 0), and its equation carries the pseudo-force moment of
 * Eq. newtonseldg, -mass cg_offset cos(alpha1 + theta) X1'' - (inertia + mass hinge_offset cg_offset cos theta)
 * alpha1'' - mass hinge_offset cg_offset sin theta alpha1'^2, with inertia about the hinge, mass >= 0 and
 * cg_offset (L2) the distance of its centre of mass from the hinge.  driver = 0: a fixed hinge.
 * All bodies of one context must use the same ds (the surface-stress regularisation weight). */
typedef struct {
  int type;
  int n_pts;
  double ds;
  double hinge[2];
  double theta0, theta_init, phi_init;
  double inertia, damping, stiffness;
  const double* pts;
  const double* ur;
  double mass_per_length, bending_stiffness, stretching_stiffness; /* DEFORMABLE only */
  double kinematics[5];   /* DRIVEN: A0, beta, sigma_t, sigma_r, f */
  double s_lo;            /* DRIVEN: position of point 0 along the plate from the reference point */
  int driver;             /* TORSIONAL: 0 fixed hinge; k > 0 hinged on the DRIVEN body k - 1 */
  double hinge_offset, mass, cg_offset; /* TORSIONAL with a driver: L1, plate mass, L2 */
  int append_to_subdomain; /* RIGID: nonzero appends the (fixed) points to Omega_0 (Sec. 3.1.1): they are
                              interpolated with E itself and get their own rows and columns in B0 (one
                              finest-level solve per appended unknown at fsi_precompute, in the context's
                              precision).  Points must lie >= 2 cells inside the grid (else
                              FSI_ERR_BODY_OUTSIDE_SUBDOMAIN at fsi_precompute), anywhere relative to the box.
                              Dense operator only: with drop_tol > 0, fsi_save_operator or fsi_load_operator
                              FSI_ERR_UNSUPPORTED.  Ignored with coupling 1. */
} fsi_body_desc;

typedef struct {
  double x_lo, x_hi, y_lo, y_hi;
} fsi_box;

typedef struct {
  int64_t steps_done;
  int last_iters;      /* FSI iterations of the last step */
  int max_iters_seen;  /* largest FSI iteration count so far */
  int n_sd;            /* number of Omega_0 points (2*n_sd unknowns) */
  int nf;              /* number of surface-stress unknowns (2 x body points) */
  double b0_seconds;   /* wall time of the last fsi_precompute */
  size_t device_bytes; /* device memory held by the context */
  int launches_per_step; /* kernels this library launches per time step (coupling 1: of the last step,
                            the loops' launches counted from the device's iteration counters) */
  int last_solves;       /* refinement solves of the small system in the last step (all FSI iterations) */
  int inverse_rebuilds;  /* times the float inverse of the small system was rebuilt so far */
  int dst_gemm[3];       /* 1 if pass p (0 forward x, 1 y solve, 2 inverse x) runs as a tensor-core GEMM */
  double dst_us[2][3];   /* autotuner timings in microseconds: [0] FFT, [1] GEMM, per pass (0 = not timed) */
  int last_refreshes;    /* Newton-Schulz refreshes of the float inverse in the last step */
  int64_t b0_nnz;        /* stored nonzero entries of B0: (2 n_sd)^2 dense, the kept entries of B0' sparse */
  int b0_window;         /* sparse B0': half-width (Omega_0 points) of each column's window; 0 dense */
  int last_krylov_iters;     /* coupling 1: Krylov iterations of the last step (all FSI iterations) */
  int64_t krylov_iters_total; /* coupling 1: Krylov iterations since the context was created */
} fsi_stats;

typedef struct fsi_ctx fsi_ctx;

/* Human-readable name of a status code (static string). */
const char* fsi_status_string(int status);
/* Text of the last CUDA error recorded by this thread (static buffer). */
const char* fsi_last_error_message(void);

/* Create a context: allocates the per-level vorticity/streamfunction fields and transform buffers on the
 * current device.  Fields start at zero (impulsive start).  *out receives the handle. */
fsi_status fsi_create(const fsi_grid_desc* grid, const fsi_exec_desc* exec, fsi_ctx** out);

/* Add a body (Sec. 2.1, App. A).  Host arrays are copied.  Must precede fsi_precompute. */
fsi_status fsi_add_body(fsi_ctx* ctx, const fsi_body_desc* body, int* body_id);

/* Fix the sub-domain Omega_0 (Sec. 3.1.1): the box is snapped to level-0 vertices at spacing h and clipped
 * to vertices at least 2 cells from the boundary.  Exactly one box and no extra points are supported
 * (n_boxes == 1, n_extra == 0; otherwise FSI_ERR_UNSUPPORTED). */
fsi_status fsi_set_subdomain(fsi_ctx* ctx, const fsi_box* boxes, int n_boxes, const double* extra_pts,
                             int n_extra);

/* Offline stage (Algorithm 1): build B0 (2 n_sd x 2 n_sd, double) on the device.
 * drop_tol = 0: the dense operator.  0 < drop_tol < 1: the sparse B0' of Eq. filtereq (the paper uses 0.007),
 * entry (i, j) kept when |b_ij| > drop_tol |b_jj| (the column's own diagonal), stored per column as a window
 * of (2w+1)^2 Omega_0 points around the column's point (w: the largest extent of a kept entry, found by a
 * scan; fsi_stats.b0_window, .b0_nnz); the small system then uses B0' and is not symmetric.  The sparse
 * operator is built from the lattice Green's function only (b0_method 0; method 1 returns
 * FSI_ERR_UNSUPPORTED).  drop_tol < 0, >= 1 or NaN: FSI_ERR_INVALID_ARG. */
fsi_status fsi_precompute(fsi_ctx* ctx, double drop_tol);

/* Save the operator built by fsi_precompute (dense B0 or the filtered B0') to the file at path (host byte
 * order; a header with the grid, Omega_0, Re, dt and drop tolerance, then the doubles).  The operator depends
 * only on those, not on the bodies, so it can be reused by later runs (see fsi_load_operator).  Before
 * fsi_precompute: FSI_ERR_STATE; coupling 1 (no operator): FSI_ERR_UNSUPPORTED; file errors:
 * FSI_ERR_INVALID_ARG (fsi_last_error_message says which).  Synchronising. */
fsi_status fsi_save_operator(fsi_ctx* ctx, const char* path);

/* Offline stage from a file written by fsi_save_operator, in place of fsi_precompute: the file's grid (nx, ny,
 * h), Omega_0 vertex box, Re and dt must equal this context's exactly (else FSI_ERR_INVALID_ARG, as for a
 * missing or truncated file); the operator's format (dense or filtered) is the file's.  Bodies are set up as
 * by fsi_precompute.  coupling 1: FSI_ERR_UNSUPPORTED. */
fsi_status fsi_load_operator(fsi_ctx* ctx, const char* path);

/* Checkpoint of a run (synchronising): the fields and previous advection term of every level, the body and
 * flag state, the last surface stress, the float inverse of the small system with its control words, the
 * interpolation map of the last step, the history ring and the step counters -- everything the next step
 * reads.  fsi_load_state restores it into a context set up the same way (same grid, precision, coupling,
 * bodies and history capacity; after its offline stage): n steps, save, load, n steps then equal 2n steps
 * bit for bit.  A file of another shape, a missing or a truncated file: FSI_ERR_INVALID_ARG, and the
 * context is left unchanged.  Before the offline stage (with bodies): FSI_ERR_STATE. */
fsi_status fsi_save_state(fsi_ctx* ctx, const char* path);
fsi_status fsi_load_state(fsi_ctx* ctx, const char* path);

/* Online stage (Algorithm 2): enqueue n_steps time steps on the context stream.  Asynchronous. */
fsi_status fsi_advance(fsi_ctx* ctx, int n_steps);

/* Wait for the context stream and return the latched device status. */
fsi_status fsi_sync(fsi_ctx* ctx);

/* Outputs of the last completed step for one body (synchronising).  fx, fy = ds * sum of the surface
 * stress (force by the fluid on the body; c_d = 2 fx, c_l = 2 fy at unit density, speed and chord);
 * moment = ds * S f about the hinge (0 for rigid and deformable bodies).  Any output pointer may be NULL.
 * fsi_get_deflection: theta, phi of a torsional body; tip displacement and its rate for a deformable one;
 * 0 for a rigid one. */
fsi_status fsi_get_forces(fsi_ctx* ctx, int body, double* fx, double* fy, double* moment);
fsi_status fsi_get_deflection(fsi_ctx* ctx, int body, double* theta, double* phi);

/* The same outputs of every body, read without waiting (the per-step read of a running job: the outputs of
 * Algorithm 2's step, as above).  Enqueues on the context stream, behind the steps enqueued so far, copies
 * into out[5 b + 0 .. 4] = fx, fy, moment, theta, phi of body b (theta, phi as fsi_get_deflection) for every
 * body b; cap = capacity of out in values, at least 5 * (number of bodies).  The values are in place once the
 * stream has passed the copies (after fsi_sync, or an event the caller records on the stream after this
 * call); the caller owns out and keeps it alive until then.  For the call to return before the steps have
 * run, out must be page-locked host memory (cudaHostAlloc or cudaHostRegister); with pageable memory the
 * CUDA runtime finishes the copy before it returns.  The device status of the steps is not read here
 * (fsi_sync returns it).  Errors: FSI_ERR_INVALID_ARG (NULL context or out, no bodies, cap too small);
 * FSI_ERR_CUDA if the copy cannot be enqueued. */
fsi_status fsi_read_outputs_async(fsi_ctx* ctx, double* out, int cap);

/* State of a DEFORMABLE body after the last completed step (synchronising): chi = node positions and
 * rotations (x, y, theta) of nodes 1..n_pts-1 (3*(n_pts-1) values, node-major), zeta = their rates,
 * zetadot = their second derivatives.  cap = capacity of each non-NULL output array in values;
 * *n_dof receives 3*(n_pts-1).  Other body types: FSI_ERR_INVALID_ARG. */
fsi_status fsi_get_beam_state(fsi_ctx* ctx, int body, double* chi, double* zeta, double* zetadot, int cap,
                              int* n_dof);

/* Per-step history of one body: field 0 fx, 1 fy, 2 moment, 3 theta, 4 phi, 5 FSI iterations.
 * Copies the last min(cap, kept) steps, oldest first; *n receives the count (synchronising). */
fsi_status fsi_get_history(fsi_ctx* ctx, int body, int field, double* out, int cap, int* n);

/* Copy a vertex field of one level to the host as double, row-major [(ny+1) x (nx+1)], boundary ring
 * included.  which: 0 = vorticity, 1 = streamfunction. */
fsi_status fsi_get_field(fsi_ctx* ctx, int level, int which, double* out);
/* Overwrite a vertex field (same layout) from the host, e.g. to start from a given state. */
fsi_status fsi_set_field(fsi_ctx* ctx, int level, int which, const double* in);

/* Sampled entries of B0 (or of the sparse B0', zero where dropped): out[k] = B0[rows[k], cols[k]] for
 * k < n (synchronising).  Unknown ordering: the n_sd x-components (points row by row inside the box),
 * then the n_sd y-components.  coupling 1 (no B0): FSI_ERR_UNSUPPORTED. */
fsi_status fsi_get_operator_entries(fsi_ctx* ctx, const int64_t* rows, const int64_t* cols, int n,
                                    double* out);

/* Double-precision Cholesky factor L L^T = B0 + tau I of the precomputed sub-domain matrix, with
 * tau = tau_rel * max_i B0_ii (B0 at flow-grid spacing is only positive semi-definite; the b0_1024 workload
 * asks for this factor after the B0 assembly).  The factor (lower triangle, 8 (2 n_sd)^2 bytes) is kept on
 * the device.  *tau_out and *seconds (wall time of the factorisation) may be NULL.  A non-positive pivot
 * returns FSI_ERR_NONFINITE.  Requires fsi_precompute with the dense operator (sparse: FSI_ERR_UNSUPPORTED). */
fsi_status fsi_factor_operator(fsi_ctx* ctx, double tau_rel, double* tau_out, double* seconds);
/* Sampled entries of that factor: out[k] = L[rows[k], cols[k]] (zero above the diagonal). */
fsi_status fsi_get_factor_entries(fsi_ctx* ctx, const int64_t* rows, const int64_t* cols, int n, double* out);

/* Interpolation map P of the last step's final FSI iterate (Eq. weights): for each body point p the four
 * Omega_0 point indices idx[4p..4p+3] and hat weights w[4p..4p+3] (synchronising).  coupling 1 (no P):
 * FSI_ERR_UNSUPPORTED. */
fsi_status fsi_get_interp(fsi_ctx* ctx, int64_t* idx, double* w, int cap_points);

fsi_status fsi_get_stats(fsi_ctx* ctx, fsi_stats* out);

/* The small system K of the last FSI iteration (Eq. stress2: (ds/h^2) P B0 P^T plus the structural terms of
 * the bodies; unknown ordering: the x-components of all body points in body order, then the y-components),
 * row-major nf x nf doubles into out (cap >= nf*nf values; *nf_out receives nf; synchronising).  With the
 * dense B0 and no deformable body K is symmetric; a deformable body's FP32 structural columns and the sparse
 * B0' make it symmetric only to rounding, or not at all.  coupling 1 or before the first step (no K):
 * FSI_ERR_STATE; cap too small: FSI_ERR_INVALID_ARG. */
fsi_status fsi_get_small_system(fsi_ctx* ctx, double* out, int64_t cap, int* nf_out);

/* Failure-detection hook (not part of the method): the FSI kernel's cross-CTA wait of the warps that assemble
 * the small system while the flags are linearised (used with DEFORMABLE bodies) polls a global arrival
 * counter a bounded number of times and latches FSI_ERR_TIMEOUT when the bound is reached.  This sets the
 * bound (polls of about 64 ns; 0 restores the default, about 4 M polls) and a number of arrivals the wait
 * requires beyond the kernel's own (0 in normal runs; > 0 makes every such wait run out, as if CTAs had
 * stopped arriving, without any fault).  Takes effect from the next step (a captured step graph is
 * rebuilt).  missing_arrivals outside [0, 1024]: FSI_ERR_INVALID_ARG.  Synchronising. */
fsi_status fsi_debug_set_wait_limit(fsi_ctx* ctx, unsigned spin_limit, int missing_arrivals);

/* Tracing: accumulated wall time (ms) of the phases of the FSI-iteration kernel since the context was
 * created, measured on the device: 0 body points / P / right-hand side, 1 assembly of P B0 P^T, 2 refresh
 * of the float inverse, 3 rebuild of the float inverse, 4 refinement solves, 5 double residuals,
 * 6 dtheta and convergence, 7 outputs; a finer split of 2, 4 and 5: 8 columns of X K, 9 rows of the new
 * X, 10 reload of X, 11 d = X r, 12 residual rows and barrier, 13 residual gather; inside 0, measured on
 * their own threads: 14 the body points (warps 0-3), 15 the linearisation and solves of the flags (warps 4-7),
 * and with flags the steps of 0 on thread 0: 16 wait for every CTA's points, 17 point tables into shared
 * memory, 18 owned rows of P B0 P^T, 19 wait for the flags' warps, 20 flags' term and publication of the rows,
 * 21 grid barrier, 22 right-hand side; 23 the owned rows of d = X r and their barrier (distributed variant;
 * 11 is then the update of f).  out[0..n-1] (n <= 24 meaningful; synchronising). */
fsi_status fsi_get_phase_times(fsi_ctx* ctx, double* out, int n);
/* Phase timers of the FSI kernel on (nonzero: the counters read by fsi_get_phase_times are cleared and the
 * steps that follow are timed) or off (the default: the timers' reads of the global timer sit in every
 * step, about 1 % of the kernel's time).  Synchronising; a captured step is captured again. */
fsi_status fsi_set_phase_timing(fsi_ctx* ctx, int on);

/* Live timing of one kernel class: runs n_steps (1..1024) ordinary time steps without a graph, records a
 * CUDA event pair on the context stream around every launch of that class and returns the mean launch
 * duration in ms and the number of timed launches.  The steps advance the simulation like fsi_advance.
 * Classes: 1 forward-x DST pass, 2 y-solve DST pass, 3 inverse-x DST pass, 4 FSI iteration kernel,
 * 5 advection/right-hand side (with the fine-to-coarse injection), 6 corrector source, 7 level boundary
 * with its side transforms. */
fsi_status fsi_profile_kernel(fsi_ctx* ctx, int kernel_class, int n_steps, double* avg_ms, int* launches);

/* Free all device memory and the handle (synchronises the stream first). */
void fsi_destroy(fsi_ctx* ctx);

/* ---- Offline stage for several independent sub-domains on one grid ------------------------------------
 * B0 (Algorithm 1, Eq. action; finest level, zero boundary values) for n_boxes Omega_0 boxes of different
 * sizes on the same grid, built together: every kernel of the build runs once over all boxes (one lattice
 * Green's function shared by all boxes with exec->b0_method = 0; batches of column solves that mix the
 * boxes' columns with b0_method = 1).  Each box is snapped and clipped as in fsi_set_subdomain.  The
 * matrices stay on the device, box k's (2 n_sd_k)^2 row-major block after box k-1's; the unknown
 * ordering inside a box is that of fsi_get_operator_entries.  exec->precision selects the arithmetic of the
 * column solves (B0 is stored in double); exec->stream as in fsi_create.  The call synchronises. */
typedef struct fsi_b0_set fsi_b0_set;

fsi_status fsi_b0_set_build(const fsi_grid_desc* grid, const fsi_exec_desc* exec, const fsi_box* boxes,
                            int n_boxes, fsi_b0_set** out);
/* Snapped extent of box k: vertex indices [i_lo, i_hi] x [j_lo, j_hi] and n_sd = points in the box.
 * Any output pointer may be NULL. */
fsi_status fsi_b0_set_box(const fsi_b0_set* set, int box, int* i_lo, int* i_hi, int* j_lo, int* j_hi, int* n_sd);
/* Sampled entries of box k's matrix: out[m] = B0_k[rows[m], cols[m]] (synchronising). */
fsi_status fsi_b0_set_entries(fsi_b0_set* set, int box, const int64_t* rows, const int64_t* cols, int n,
                              double* out);
/* Wall time of the build in seconds and device bytes held by the set.  Either pointer may be NULL. */
fsi_status fsi_b0_set_stats(const fsi_b0_set* set, double* seconds, size_t* device_bytes);
void fsi_b0_set_destroy(fsi_b0_set* set);

#ifdef __cplusplus
}
#endif
#endif /* IBFSI_H */
