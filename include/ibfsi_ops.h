/*
 * ibfsi_ops.h -- operator-level entry points of the GB300 sub-domain IB-FSI library, for testing and
 * measuring single stages of the hot path in isolation.  Same conventions as ibfsi.h: host pointers,
 * inputs copied, caller owns every buffer, status codes instead of aborts.
 */
#ifndef IBFSI_OPS_H
#define IBFSI_OPS_H

#include "ibfsi.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One DST-diagonalised solve on a single level with zero boundary values (Sec. 3.2.1, Eq. predictor2):
 * w = A_w^{-1} rhs with A_w = 1/dt - lap_h/(2 re), then s = (-lap_h)^{-1} w.
 * rhs: interior values, row-major [(ny-1) x (nx-1)] (rows = y).  w_out, s_out: same layout.
 * precision: FSI_PREC_FP64 or FSI_PREC_FP32 (inputs/outputs are double either way).
 * nx, ny: cell counts as in a grid descriptor, 2^k or 3 * 2^k in [16, 2048]; h, re, dt > 0.  Runs on the current device,
 * synchronously. */
fsi_status fsi_op_level_solve(int precision, int nx, int ny, double h, double re, double dt, const double* rhs,
                              double* w_out, double* s_out);

/* The same solve with a choice of sine-transform implementation (fsi_exec_desc.dst_method): 0 FFT passes,
 * 1 tensor-core sine-matrix GEMMs (FP32 only, nx in [128, 1024], ny in [128, 512]; otherwise FSI_ERR_UNSUPPORTED),
 * 2 autotuned per pass. */
fsi_status fsi_op_level_solve_ex(int precision, int dst_method, int nx, int ny, double h, double re, double dt,
                                 const double* rhs, double* w_out, double* s_out);

/* Allocation-free variant of fsi_op_level_solve for callers that cannot call cudaMalloc (for example code
 * running under a framework whose allocator owns all device memory, or a callback that must not allocate).
 * The paper has no counterpart: this is a service of this library.
 * Same solve (zero boundary values), but inputs and outputs are DEVICE pointers supplied by the caller and
 * the work is enqueued on `stream` (cudaStream_t; NULL = legacy default stream) without synchronising:
 *   rhs_dev  [(ny-1) x (nx-1)] interior right-hand side, row-major, float (FP32) or double (FP64);
 *   w_dev, s_dev  [(ny+1) x (nx+1)] vertex arrays of the same type: interior entries are overwritten, the
 *                 boundary ring is left as it is.
 * Scratch lives in a fixed 8 MiB device array inside the library (held by every device that loads it):
 * sizes needing more -- e.g. FP64 above 512 x 512, FP32 above 1024 x 512 -- return FSI_ERR_UNSUPPORTED with
 * the reason in fsi_last_error_message.  No device memory is allocated or freed by this call.
 * The first call on a device takes the scratch address (cudaGetSymbolAddress) and sets kernel attributes;
 * make that first call before any stream capture.  The address and attributes are cached per device for the
 * life of the process: after cudaDeviceReset (or any teardown of the device's primary context) they are
 * stale, so do not call this entry point again in that process.  All calls share the scratch array: calls whose work
 * overlaps on the GPU race and must be ordered by the caller (one stream, or events). */
fsi_status fsi_op_level_solve_noalloc(int precision, int nx, int ny, double h, double re, double dt,
                                      const void* rhs_dev, void* w_dev, void* s_dev, void* stream);

/* Throughput of a project-written fused multiply-add loop on the current device (independent chains, all
 * SMs busy), used as the arithmetic roofline of the FP64 and FP32 paths.  *flops_per_s receives the
 * measured rate (2 flops per FMA).  precision: FSI_PREC_FP64 or FSI_PREC_FP32. */
fsi_status fsi_op_fma_rate(int precision, double* flops_per_s);

/* The structural linearisation of a deformable body as the FSI kernel runs it (Eq. beam; App. A with
 * J_d = 4M/dt^2 + K(chi); the element, mass and state conventions of the DEFORMABLE body in ibfsi.h), in one
 * GPU launch: for a flag of n_el elements of length ds clamped at (cx, cy),
 *   r_zeta = M ((4/dt^2)(chi_n - chi) + (4/dt) zeta_n + zetadot_n) - R(chi)      (FP64)
 *   x = J_d(chi)^-1 b                                                           (J_d factored in FP32)
 * chi, chi_n, zeta_n, zetadot_n, b, r_zeta, x: 3*n_el doubles (x, y, theta of nodes 1..n_el);
 * ref: per element psi, c, s of a reference chord from which the element's rotation is measured (3*n_el
 * doubles; the chord at chi_n, psi measured from the undeformed direction).  Host pointers; r_zeta or x may
 * be NULL.  n_el in [1, 1000]; mu, ei, ea, ds, dt > 0.  Runs on the current device, synchronously. */
fsi_status fsi_op_beam_solve(int n_el, double ds, double mu, double ei, double ea, double cx, double cy,
                             double dt, const double* chi, const double* chi_n, const double* zeta_n,
                             const double* zetadot_n, const double* ref, const double* b, double* r_zeta,
                             double* x);

/* The prescribed kinematics of a DRIVEN plate (Sec. 5.1; the formulas of the DRIVEN body in ibfsi.h) as the
 * library evaluates them on the host for every step: out = {X1, X1', X1'', alpha1, alpha1', alpha1''} at
 * time t (derivatives in t), G_t by composite 16-point Gauss-Legendre quadrature over 16 panels of the
 * fractional period.  params = {A0, beta, sigma_t, sigma_r, f} (host, 5 doubles); out: host, 6 doubles.
 * Host computation only: no GPU is used.  Invalid params (A0 < 0, sigma or f <= 0, non-finite values):
 * FSI_ERR_INVALID_ARG. */
fsi_status fsi_op_flapping_kinematics(const double* params, double t, double* out);

#ifdef __cplusplus
}
#endif
#endif /* IBFSI_OPS_H */
