// True-E coupling (Sec. 2.2): the comparator of Sec. 5.1 that the sub-domain method is measured against.
//
// Each FSI iteration (Eqs. stress2, dtheta2, with E and E^T evaluated at the body points of the iterate)
// solves
//   ( (ds/h^2) E C (C^T A C)^-1 C^T E^T + sum_b (2 ds/dt)/J_b S_b S_b^T ) f = r^c(k)
// without forming the matrix.  The paper runs GMRES with one (C^T A C)^-1 per Krylov iteration (Sec. 3, the
// bottleneck the sub-domain method removes); the operator is symmetric positive definite, so conjugate
// gradients reach the same unique solution, also with one (C^T A C)^-1 per iteration.  One CG iteration:
//   k_te_src  -- E^T p spread onto the faces and its curl, on the vertex box of Omega_0 grown by 3 cells
//                (Omega_0 holds the range of motion, so the support never leaves the box);
//   the three sine-transform passes of the finest level with homogeneous boundary values (as the
//                corrector);
//   k_te_cg   -- E C s at the body points, the structural rank-one terms, the CG update (one CTA).
// The FSI and CG loops run on the device as CUDA-graph WHILE nodes whose conditions the kernels set (a step
// needs no host round trip); eager steps read the same flags on the host after each iteration.  Every loop is
// bounded by an iteration counter that the kernel setting its condition increments.
#include <cmath>
#include "internal.h"

namespace {

constexpr int kThr = 512;  // threads of the one-CTA kernels

// 4 x 4 face window of one body point for each velocity component: u faces (iu + d, ju + e) at
// (x_{iu+d}, y_{ju+e+1/2}), v faces (iv + d, jv + e) at (x_{iv+d+1/2}, y_{jv+e}); weight wx[d] * wy[e].
struct TePoint {
  int iu, ju, iv, jv;
  double wxu[4], wyu[4], wxv[4], wyv[4];
};

// control words
enum { TC_CG_IT = 0, TC_CG_DONE, TC_FSI_IT, TC_FSI_DONE, TC_CG_STEP, TC_CG_LAST, TC_N };
// scalars: 0 r.r, 1 threshold on r.r
enum { TS_RR = 0, TS_THR, TS_N };

struct TeArgs {
  const void* s0;  // level-0 streamfunction after the predictor (s*), context precision
  const void* ts;  // level-0 streamfunction of the operator application
  int fp64;
  long ps;
  double x0, y0, h, dt, ds, U, V, tol, ktol, two_dt, four_dt2, kscale;  // kscale = ds / h^2
  int max_iters, kmax;
  int nb, nf, n_bodies;
  int i_lo, i_hi, j_lo, j_hi;  // Omega_0 vertex box: every body point must lie inside
  const BodyDev* bodies;
  BodyState* st;
  const int* point_body;
  const double* rpts;
  const double* rur;
  TePoint* pt;
  double *f, *r, *p, *rhs, *sv;
  double* scal;
  int* ctl;
  unsigned long long* cg_total;
  int* status;
  int* ctrl;
  double* hist;
  int hist_cap;
  cudaGraphConditionalHandle h_fsi, h_cg;
  int use_cond;
};

__device__ __forceinline__ double load_s(const void* s, int fp64, long o) {
  return fp64 ? ((const double*)s)[o] : (double)((const float*)s)[o];
}

// deterministic block sum (every thread receives the result)
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// 3-point discrete delta in grid units (Sec. 2.2, reading R1); explicit roundings (no contraction).
__device__ double delta3(double r) {
  r = fabs(r);
  if (r <= 0.5) return __ddiv_rn(__dadd_rn(1.0, sqrt(__dsub_rn(1.0, __dmul_rn(3.0, __dmul_rn(r, r))))), 3.0);
  if (r <= 1.5) {
    const double a = __dsub_rn(1.0, r);
    const double q = fmax(0.0, __dsub_rn(1.0, __dmul_rn(3.0, __dmul_rn(a, a))));
    return __ddiv_rn(__dsub_rn(__dsub_rn(5.0, __dmul_rn(3.0, r)), sqrt(q)), 6.0);
  }
  return 0.0;
}

// window of the faces offset (ox, oy) cells from the vertices, around the point at grid coordinates (X, Y)
__device__ void face_window(double X, double Y, double ox, double oy, int* i0, int* j0, double* wx, double* wy) {
  const int a = (int)floor(X - ox) - 1, b = (int)floor(Y - oy) - 1;
  *i0 = a;
  *j0 = b;
  for (int d = 0; d < 4; ++d) {
    wx[d] = delta3(__dsub_rn(__dadd_rn((double)(a + d), ox), X));
    wy[d] = delta3(__dsub_rn(__dadd_rn((double)(b + d), oy), Y));
  }
}

// ---------------------------------------------------------------------------------------------------------
// Start of an FSI iteration: body points of the iterate, their face windows, S, the right-hand side
// r^c(k) = E (C s* + q_inf) - u_rigid - S phi^(k) + S (r^theta(k) - (2/dt) r^phi(k) / J), and the CG start
// from the current f.  On the first iteration of a step the structural terms of the step are set up.
__global__ void __launch_bounds__(kThr) k_te_prep(TeArgs a) {
  const int tid = threadIdx.x, nb = a.nb;
  if (a.ctl[TC_FSI_IT] == 0) {
    for (int bi = tid; bi < a.n_bodies; bi += kThr) {
      const BodyDev b = a.bodies[bi];
      BodyState& s = a.st[bi];
      if (b.type == FSI_BODY_TORSIONAL) {
        const double dt = a.dt;
        s.jac = 4.0 * b.inertia / (dt * dt) + 2.0 * b.damping / dt + b.stiffness;
        s.r_phi = b.inertia * (4.0 * s.theta / (dt * dt) + 4.0 * s.phi / dt + s.phidot) +
                  b.damping * (2.0 * s.theta / dt + s.phi);
        s.r_theta = s.phi + 2.0 / dt * s.theta;
      }
      s.theta_k = s.theta;
      s.phi_k = s.phi;
      s.theta_p = s.theta;
    }
    __syncthreads();
  }
  for (int p = tid; p < nb; p += kThr) {
    const int bi = a.point_body[p];
    const BodyDev b = a.bodies[bi];
    double x, y, svx = 0.0, svy = 0.0, ux = 0.0, uy = 0.0;
    if (b.type == FSI_BODY_TORSIONAL) {
      const BodyState s = a.st[bi];
      double sn, cs;
      sincos(b.theta0 + s.theta_k, &sn, &cs);
      const double q = (double)(p - b.off) * a.ds;
      x = __dadd_rn(b.hx, __dmul_rn(q, cs));
      y = __dadd_rn(b.hy, __dmul_rn(q, sn));
      svx = q * (-sn);
      svy = q * cs;
      const double rphik = s.r_phi - s.jac * s.theta_k;
      const double rthk = s.r_theta - a.two_dt * s.theta_k + s.phi_k;
      const double coef = rthk - a.two_dt * rphik / s.jac;
      ux = svx * s.phi_k - svx * coef;
      uy = svy * s.phi_k - svy * coef;
    } else {
      x = a.rpts[2 * p];
      y = a.rpts[2 * p + 1];
      ux = a.rur[2 * p];
      uy = a.rur[2 * p + 1];
    }
    double X = (x - a.x0) / a.h, Y = (y - a.y0) / a.h;
    if (!(X >= (double)a.i_lo && X <= (double)a.i_hi && Y >= (double)a.j_lo && Y <= (double)a.j_hi)) {
      dev_set_status(a.status, FSI_ERR_BODY_OUTSIDE_SUBDOMAIN);
      X = fmin(fmax(isfinite(X) ? X : (double)a.i_lo, (double)a.i_lo), (double)a.i_hi);
      Y = fmin(fmax(isfinite(Y) ? Y : (double)a.j_lo, (double)a.j_lo), (double)a.j_hi);
    }
    TePoint P;
    face_window(X, Y, 0.0, 0.5, &P.iu, &P.ju, P.wxu, P.wyu);
    face_window(X, Y, 0.5, 0.0, &P.iv, &P.jv, P.wxv, P.wyv);
    a.pt[p] = P;
    // E (C s* + q_inf): u = (s[J+1][I] - s[J][I]) / h + U on u faces, v = -(s[J][I+1] - s[J][I]) / h + V
    double eu = 0.0, ev = 0.0;
    for (int e = 0; e < 4; ++e)
      for (int d = 0; d < 4; ++d) {
        const long I = P.iu + d, J = P.ju + e;
        const double u = (load_s(a.s0, a.fp64, (J + 1) * a.ps + I) - load_s(a.s0, a.fp64, J * a.ps + I)) / a.h + a.U;
        eu = __dadd_rn(eu, __dmul_rn(__dmul_rn(P.wxu[d], P.wyu[e]), u));
      }
    for (int e = 0; e < 4; ++e)
      for (int d = 0; d < 4; ++d) {
        const long I = P.iv + d, J = P.jv + e;
        const double v = -(load_s(a.s0, a.fp64, J * a.ps + I + 1) - load_s(a.s0, a.fp64, J * a.ps + I)) / a.h + a.V;
        ev = __dadd_rn(ev, __dmul_rn(__dmul_rn(P.wxv[d], P.wyv[e]), v));
      }
    a.rhs[p] = eu - ux;
    a.rhs[nb + p] = ev - uy;
    a.sv[p] = svx;
    a.sv[nb + p] = svy;
  }
  for (int k = tid; k < a.nf; k += kThr) a.p[k] = a.f[k];  // the first application is K f (CG start)
  if (tid == 0) {
    a.ctl[TC_CG_IT] = 0;
    a.ctl[TC_CG_DONE] = 0;
    if (a.use_cond) cudaGraphSetConditional(a.h_cg, 1u);
  }
}

// curl of E^T v (scaled by pre) at the interior vertices of the box [wi0, wi1] x [wj0, wj1]:
// src(i, j) = pre ((Fv(i+1/2, j) - Fv(i-1/2, j)) / h - (Fu(i, j+1/2) - Fu(i, j-1/2)) / h), where the face
// values F sum w f over the points in point order.  Threads of a 32 x 4 tile, one vertex each.
template <typename T>
__global__ void __launch_bounds__(128) k_te_src(T* __restrict__ src, long ps, int wi0, int wi1, int wj0, int wj1,
                                                const TePoint* __restrict__ pt, const double* __restrict__ vec,
                                                int nb, double h, double pre) {
  extern __shared__ __align__(16) unsigned char te_smem[];
  TePoint* sp = reinterpret_cast<TePoint*>(te_smem);
  double* sf = reinterpret_cast<double*>(sp + nb);
  for (int k = threadIdx.x; k < nb; k += 128) sp[k] = pt[k];
  for (int k = threadIdx.x; k < 2 * nb; k += 128) sf[k] = vec[k];
  __syncthreads();
  const int i = wi0 + (int)blockIdx.x * 32 + (threadIdx.x & 31);
  const int j = wj0 + (int)blockIdx.y * 4 + (threadIdx.x >> 5);
  if (i > wi1 || j > wj1) return;
  double fun = 0.0, fus = 0.0, fve = 0.0, fvw = 0.0;
  for (int q = 0; q < nb; ++q) {
    const TePoint& P = sp[q];
    const int du = i - P.iu;
    if (du >= 0 && du < 4) {
      const double fx = sf[q];
      const int en = j - P.ju, es = j - 1 - P.ju;
      if (en >= 0 && en < 4) fun = __dadd_rn(fun, __dmul_rn(__dmul_rn(P.wxu[du], P.wyu[en]), fx));
      if (es >= 0 && es < 4) fus = __dadd_rn(fus, __dmul_rn(__dmul_rn(P.wxu[du], P.wyu[es]), fx));
    }
    const int ev = j - P.jv;
    if (ev >= 0 && ev < 4) {
      const double fy = sf[nb + q];
      const int de = i - P.iv, dw = i - 1 - P.iv;
      if (de >= 0 && de < 4) fve = __dadd_rn(fve, __dmul_rn(__dmul_rn(P.wxv[de], P.wyv[ev]), fy));
      if (dw >= 0 && dw < 4) fvw = __dadd_rn(fvw, __dmul_rn(__dmul_rn(P.wxv[dw], P.wyv[ev]), fy));
    }
  }
  const double c = __dsub_rn(__ddiv_rn(__dsub_rn(fve, fvw), h), __ddiv_rn(__dsub_rn(fun, fus), h));
  src[(long)(j - 1) * ps + (i - 1)] = T(__dmul_rn(pre, c));
}

// One CG iteration after the operator application: q = (ds/h^2) E C s_t + sum_b kc_b S_b (S_b . p) with
// p the applied vector, then (iteration 0) r = rhs - q, p = r, or (later) the CG update of f, r and p.
// Sets the CG loop condition on every path.
__global__ void __launch_bounds__(kThr) k_te_cg(TeArgs a) {
  extern __shared__ double q[];  // [nf]
  __shared__ double red[32];
  const int tid = threadIdx.x, nb = a.nb, nf = a.nf;
  const int it = a.ctl[TC_CG_IT];
  for (int p = tid; p < nb; p += kThr) {
    const TePoint P = a.pt[p];
    double qu = 0.0, qv = 0.0;
    for (int e = 0; e < 4; ++e)
      for (int d = 0; d < 4; ++d) {
        const long I = P.iu + d, J = P.ju + e;
        const double u = (load_s(a.ts, a.fp64, (J + 1) * a.ps + I) - load_s(a.ts, a.fp64, J * a.ps + I)) / a.h;
        qu = __dadd_rn(qu, __dmul_rn(__dmul_rn(P.wxu[d], P.wyu[e]), u));
      }
    for (int e = 0; e < 4; ++e)
      for (int d = 0; d < 4; ++d) {
        const long I = P.iv + d, J = P.jv + e;
        const double v = -(load_s(a.ts, a.fp64, J * a.ps + I + 1) - load_s(a.ts, a.fp64, J * a.ps + I)) / a.h;
        qv = __dadd_rn(qv, __dmul_rn(__dmul_rn(P.wxv[d], P.wyv[e]), v));
      }
    q[p] = a.kscale * qu;
    q[nb + p] = a.kscale * qv;
  }
  __syncthreads();
  for (int bi = 0; bi < a.n_bodies; ++bi) {  // structural rank-one terms (2 ds/dt)/J S S^T p
    const BodyDev b = a.bodies[bi];
    if (b.type != FSI_BODY_TORSIONAL) continue;
    double part = 0.0;
    for (int p = b.off + tid; p < b.off + b.n; p += kThr) part += a.sv[p] * a.p[p] + a.sv[nb + p] * a.p[nb + p];
    const double dot = block_sum(part, red);
    const double kc = (2.0 * a.ds / a.dt) / a.st[bi].jac;
    for (int p = b.off + tid; p < b.off + b.n; p += kThr) {
      q[p] += kc * a.sv[p] * dot;
      q[nb + p] += kc * a.sv[nb + p] * dot;
    }
    __syncthreads();
  }
  bool done;
  if (it == 0) {
    double prr = 0.0, pbb = 0.0;
    for (int k = tid; k < nf; k += kThr) {
      const double rk = a.rhs[k] - q[k];
      a.r[k] = rk;
      a.p[k] = rk;
      prr += rk * rk;
      pbb += a.rhs[k] * a.rhs[k];
    }
    const double rr = block_sum(prr, red), bb = block_sum(pbb, red);
    const double thr = a.ktol * a.ktol * (bb > 0.0 ? bb : rr);
    done = !(rr > thr);
    if (tid == 0) {
      a.scal[TS_RR] = rr;
      a.scal[TS_THR] = thr;
    }
  } else {
    double ppq = 0.0;
    for (int k = tid; k < nf; k += kThr) ppq += a.p[k] * q[k];
    const double pq = block_sum(ppq, red);
    const double rr = a.scal[TS_RR];
    const double alpha = rr / pq;
    double prr = 0.0;
    for (int k = tid; k < nf; k += kThr) {
      a.f[k] += alpha * a.p[k];
      const double rk = a.r[k] - alpha * q[k];
      a.r[k] = rk;
      prr += rk * rk;
    }
    const double rn = block_sum(prr, red);
    const double beta = rn / rr;
    for (int k = tid; k < nf; k += kThr) a.p[k] = a.r[k] + beta * a.p[k];
    done = !(pq > 0.0) || !(rn > a.scal[TS_THR]);
    __syncthreads();
    if (tid == 0) a.scal[TS_RR] = rn;
  }
  if (tid == 0) {
    const int n = it + 1;
    if (!done && n >= a.kmax) {
      dev_set_status(a.status, FSI_ERR_NOT_CONVERGED);
      done = true;
    }
    a.ctl[TC_CG_IT] = n;
    a.ctl[TC_CG_DONE] = done ? 1 : 0;
    a.ctl[TC_CG_STEP] += 1;
    if (a.use_cond) cudaGraphSetConditional(a.h_cg, done ? 0u : 1u);
  }
}

// End of an FSI iteration (Eq. dtheta2): dtheta = (r^phi(k) + ds S f) / J for every torsional body,
// convergence on max |dtheta|; sets the FSI loop condition on every path.
__global__ void __launch_bounds__(kThr) k_te_post(TeArgs a) {
  __shared__ double red[32];
  const int tid = threadIdx.x, nb = a.nb;
  double dmax = 0.0;
  bool finite = true;
  for (int bi = 0; bi < a.n_bodies; ++bi) {
    const BodyDev b = a.bodies[bi];
    if (b.type != FSI_BODY_TORSIONAL) continue;
    double part = 0.0;
    for (int p = b.off + tid; p < b.off + b.n; p += kThr) part += a.sv[p] * a.f[p] + a.sv[nb + p] * a.f[nb + p];
    const double sf = block_sum(part, red);
    BodyState& s = a.st[bi];
    const double dth = (s.r_phi - s.jac * s.theta_k + a.ds * sf) / s.jac;
    __syncthreads();
    if (tid == 0) {
      s.theta_p = s.theta_k;
      s.theta_k += dth;
      s.phi_k = a.two_dt * s.theta_k - s.r_theta;
    }
    if (!isfinite(dth)) finite = false;
    dmax = fmax(dmax, fabs(dth));
    __syncthreads();
  }
  if (tid == 0) {
    const int n = a.ctl[TC_FSI_IT] + 1;
    const bool converged = dmax <= a.tol || !finite;
    if (!finite) dev_set_status(a.status, FSI_ERR_NONFINITE);
    if (!converged && n >= a.max_iters) dev_set_status(a.status, FSI_ERR_NOT_CONVERGED);
    const bool cont = !converged && n < a.max_iters;
    a.ctl[TC_FSI_IT] = n;
    a.ctl[TC_FSI_DONE] = cont ? 0 : 1;
    if (a.use_cond) cudaGraphSetConditional(a.h_fsi, cont ? 1u : 0u);
  }
}

// Newmark update of the torsional bodies, forces, moment about the hinge (S of the final solve), history.
__global__ void __launch_bounds__(kThr) k_te_finish(TeArgs a) {
  __shared__ double red[32];
  const int tid = threadIdx.x, nb = a.nb;
  const int slot = a.ctrl[2] % a.hist_cap;
  const int iters = a.ctl[TC_FSI_IT];
  for (int bi = 0; bi < a.n_bodies; ++bi) {
    const BodyDev b = a.bodies[bi];
    double sn = 0.0, cs = 0.0;
    if (b.type == FSI_BODY_TORSIONAL) sincos(b.theta0 + a.st[bi].theta_p, &sn, &cs);
    double px = 0.0, py = 0.0, pm = 0.0;
    for (int p = b.off + tid; p < b.off + b.n; p += kThr) {
      const double fxp = a.f[p], fyp = a.f[nb + p];
      const double q = (double)(p - b.off) * a.ds;
      px += fxp;
      py += fyp;
      pm += q * (-sn) * fxp + q * cs * fyp;
    }
    const double sx = block_sum(px, red), sy = block_sum(py, red), sm = block_sum(pm, red);
    if (tid == 0) {
      BodyState& s = a.st[bi];
      s.fx = a.ds * sx;
      s.fy = a.ds * sy;
      s.moment = b.type == FSI_BODY_TORSIONAL ? a.ds * sm : 0.0;
      if (b.type == FSI_BODY_TORSIONAL) {
        const double th_new = s.theta_k;
        const double ph_new = a.two_dt * th_new - s.r_theta;
        s.phidot = a.four_dt2 * (th_new - s.theta) - 2.0 * a.two_dt * s.phi - s.phidot;
        s.theta = th_new;
        s.phi = ph_new;
        s.phi_k = ph_new;
      }
      double* hrow = a.hist + ((long)slot * a.n_bodies + bi) * 6;
      hrow[0] = s.fx;
      hrow[1] = s.fy;
      hrow[2] = s.moment;
      hrow[3] = b.type == FSI_BODY_TORSIONAL ? s.theta : 0.0;
      hrow[4] = b.type == FSI_BODY_TORSIONAL ? s.phi : 0.0;
      hrow[5] = (double)iters;
      if (!isfinite(s.fx) || !isfinite(s.fy)) dev_set_status(a.status, FSI_ERR_NONFINITE);
    }
    __syncthreads();
  }
  if (tid == 0) {
    a.ctrl[1] = iters;
    a.ctrl[2] += 1;
    a.ctl[TC_FSI_IT] = 0;
    a.ctl[TC_CG_LAST] = a.ctl[TC_CG_STEP];
    *a.cg_total += (unsigned long long)a.ctl[TC_CG_STEP];
    a.ctl[TC_CG_STEP] = 0;
  }
}

TeArgs te_args(fsi_ctx* c) {
  TeArgs a = {};
  a.s0 = c->s_all;
  a.ts = c->te_s;
  a.fp64 = c->prec == FSI_PREC_FP64;
  a.ps = c->ps;
  a.x0 = c->g.x0;
  a.y0 = c->g.y0;
  a.h = c->g.h;
  a.dt = c->g.dt;
  a.ds = c->ds;
  a.U = c->g.uinf[0];
  a.V = c->g.uinf[1];
  a.tol = c->x.tol;
  a.ktol = c->x.krylov_tol;
  a.two_dt = 2.0 / c->g.dt;
  a.four_dt2 = 4.0 / (c->g.dt * c->g.dt);
  a.kscale = c->ds / (c->g.h * c->g.h);
  a.max_iters = c->x.max_iters;
  a.kmax = c->x.krylov_max_iters;
  a.nb = c->nb;
  a.nf = c->nf;
  a.n_bodies = c->n_bodies;
  a.i_lo = c->i_lo;
  a.i_hi = c->i_hi;
  a.j_lo = c->j_lo;
  a.j_hi = c->j_hi;
  a.bodies = c->d_bodies;
  a.st = c->d_state;
  a.point_body = c->d_point_body;
  a.rpts = c->d_rpts;
  a.rur = c->d_rur;
  a.pt = (TePoint*)c->d_te_pt;
  a.f = c->d_f;
  a.r = c->d_te_r;
  a.p = c->d_te_p;
  a.rhs = c->d_rhs;
  a.sv = c->d_sv;
  a.scal = c->d_te_scal;
  a.ctl = c->d_te_ctl;
  a.cg_total = c->d_te_total;
  a.status = c->d_status;
  a.ctrl = c->d_ctrl;
  a.hist = c->d_hist;
  a.hist_cap = c->hist_cap;
  return a;
}

// curl of E^T vec (times pre) into the source buffer; the vertex box is the interior part of Omega_0 grown by
// 3 cells, which holds the support of every point inside Omega_0
template <typename T>
fsi_status launch_src(fsi_ctx* c, const double* vec, double pre) {
  const int wi0 = c->i_lo - 3 < 1 ? 1 : c->i_lo - 3, wi1 = c->i_hi + 3 > c->nx - 1 ? c->nx - 1 : c->i_hi + 3;
  const int wj0 = c->j_lo - 3 < 1 ? 1 : c->j_lo - 3, wj1 = c->j_hi + 3 > c->ny - 1 ? c->ny - 1 : c->j_hi + 3;
  const dim3 grid((wi1 - wi0 + 32) / 32, (wj1 - wj0 + 4) / 4);
  const size_t sm = (size_t)c->nb * (sizeof(TePoint) + 2 * sizeof(double));
  k_te_src<T><<<grid, 128, sm, c->stream>>>((T*)c->src, c->ps, wi0, wi1, wj0, wj1, (const TePoint*)c->d_te_pt, vec,
                                            c->nb, c->g.h, pre);
  FSI_CUDA_TRY(cudaGetLastError());
  c->launches_per_step += 1;
  return FSI_OK;
}

fsi_status launch_src_any(fsi_ctx* c, const double* vec, double pre) {
  return c->prec == FSI_PREC_FP64 ? launch_src<double>(c, vec, pre) : launch_src<float>(c, vec, pre);
}

fsi_status launch_one(fsi_ctx* c, void (*k)(TeArgs), const TeArgs& a, size_t smem) {
  k<<<1, kThr, smem, c->stream>>>(a);
  FSI_CUDA_TRY(cudaGetLastError());
  c->launches_per_step += 1;
  return FSI_OK;
}

// one CG iteration: operator application to p, then the update
fsi_status cg_iteration(fsi_ctx* c, const TeArgs& a) {
  fsi_status st = launch_src_any(c, c->d_te_p, 1.0);
  if (st != FSI_OK) return st;
  st = launch_level_solve(c, 0, c->src, c->te_w, c->te_s, 0, 0);
  if (st != FSI_OK) return st;
  return launch_one(c, k_te_cg, a, (size_t)c->nf * sizeof(double));
}

fsi_status read_flag(fsi_ctx* c, int which, int* v) {
  FSI_CUDA_TRY(cudaMemcpyAsync(v, c->d_te_ctl + which, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return FSI_OK;
}

// a conditional handle on the graph that c->stream is being captured into (value 1 when the graph is launched)
fsi_status new_handle(fsi_ctx* c, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  FSI_CUDA_TRY(cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive || !g) return FSI_ERR_CUDA;
  FSI_CUDA_TRY(cudaGraphConditionalHandleCreate(h, g, 1u, cudaGraphCondAssignDefault));
  return FSI_OK;
}

// WHILE node on handle h (created on the same graph) at the current capture position of c->stream; body()
// is captured into the node's body graph on stream `inner` (c->stream points to it meanwhile).
template <typename F>
fsi_status capture_while(fsi_ctx* c, cudaStream_t inner, cudaGraphConditionalHandle h, F&& body) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  FSI_CUDA_TRY(cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, &ed, &nd));
  if (cs != cudaStreamCaptureStatusActive || !g) return FSI_ERR_CUDA;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  FSI_CUDA_TRY(cudaGraphAddNode(&node, g, deps, ed, nd, &np));
  cudaGraph_t bg = np.conditional.phGraph_out[0];
  FSI_CUDA_TRY(cudaStreamBeginCaptureToGraph(inner, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaStream_t outer = c->stream;
  c->stream = inner;
  const fsi_status st = body();
  c->stream = outer;
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(inner, &out);
  if (st != FSI_OK) return st;
  FSI_CUDA_TRY(e);
  FSI_CUDA_TRY(cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return FSI_OK;
}

fsi_status fsi_loop_eager(fsi_ctx* c, const TeArgs& a) {
  for (int it = 0; it < c->x.max_iters; ++it) {
    fsi_status st = launch_one(c, k_te_prep, a, 0);
    if (st != FSI_OK) return st;
    for (int k = 0; k < c->x.krylov_max_iters; ++k) {
      st = cg_iteration(c, a);
      if (st != FSI_OK) return st;
      int done = 0;
      st = read_flag(c, TC_CG_DONE, &done);
      if (st != FSI_OK) return st;
      if (done) break;
    }
    st = launch_one(c, k_te_post, a, 0);
    if (st != FSI_OK) return st;
    int done = 0;
    st = read_flag(c, TC_FSI_DONE, &done);
    if (st != FSI_OK) return st;
    if (done) break;
  }
  return FSI_OK;
}

fsi_status fsi_loop_graph(fsi_ctx* c, TeArgs& a) {
  a.use_cond = 1;
  fsi_status st = new_handle(c, &a.h_fsi);
  if (st != FSI_OK) return st;
  return capture_while(c, c->te_stream[0], a.h_fsi, [&]() -> fsi_status {
    fsi_status s = new_handle(c, &a.h_cg);  // on the FSI loop's body graph, before prep (which sets it)
    if (s != FSI_OK) return s;
    s = launch_one(c, k_te_prep, a, 0);
    if (s != FSI_OK) return s;
    s = capture_while(c, c->te_stream[1], a.h_cg, [&]() -> fsi_status { return cg_iteration(c, a); });
    if (s != FSI_OK) return s;
    return launch_one(c, k_te_post, a, 0);
  });
}

}  // namespace

// FSI iteration with the true E and the corrector of one step, after the predictor.  capture != 0: the
// stream is being captured and the loops become WHILE nodes; otherwise the loops run from the host.  The
// launches of the loops are not counted in launches_per_step (their number varies; the device counters
// give it).
fsi_status launch_true_e(fsi_ctx* c, int capture) {
  TeArgs a = te_args(c);
  const int counted = c->launches_per_step;
  fsi_status st = capture ? fsi_loop_graph(c, a) : fsi_loop_eager(c, a);
  if (st != FSI_OK) return st;
  c->launches_per_step = counted;
  st = launch_src_any(c, c->d_f, c->ds / (c->g.h * c->g.h));
  if (st != FSI_OK) return st;
  st = launch_level_solve(c, 0, c->src, c->w_all, c->s_all, 0, 1);
  if (st != FSI_OK) return st;
  return launch_one(c, k_te_finish, a, 0);
}

// kernel attributes (dynamic shared memory of the source and CG kernels for nb points)
fsi_status true_e_setup(fsi_ctx* c) {
  const int src_sm = (int)((size_t)c->nb * (sizeof(TePoint) + 2 * sizeof(double)));
  FSI_CUDA_TRY(cudaFuncSetAttribute(k_te_src<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, src_sm));
  FSI_CUDA_TRY(cudaFuncSetAttribute(k_te_src<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, src_sm));
  FSI_CUDA_TRY(cudaFuncSetAttribute(k_te_cg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)((size_t)c->nf * sizeof(double))));
  return FSI_OK;
}

size_t true_e_point_bytes() { return sizeof(TePoint); }
