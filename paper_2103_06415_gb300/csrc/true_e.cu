// True-E coupling (Sec. 2.2): the comparator of Sec. 5.1 that the sub-domain method is measured against.
//
// Each FSI iteration (Eqs. stress2, dtheta2, with E and E^T evaluated at the body points of the iterate)
// solves
//   ( (ds/h^2) E C (C^T A C)^-1 C^T E^T + sum_b (2 ds/dt)/J_b S_b S_b^T ) f = r^c(k)
// without forming the matrix.  The paper runs GMRES with one (C^T A C)^-1 per Krylov iteration (Sec. 3, the
// bottleneck the sub-domain method removes); the operator is symmetric positive definite, so conjugate
// gradients reach the same unique solution, also with one (C^T A C)^-1 per iteration.  One CG iteration:
//   k_te_src   -- E^T p spread onto the faces and its curl, on the vertex box of Omega_0 grown by 3 cells
//                 (Omega_0 holds the range of motion, so the support never leaves the box);
//   the three sine-transform passes of the finest level with homogeneous boundary values (as the
//                 corrector);
//   k_te_apply -- (ds/h^2) E C s at the body points (several CTAs);
//   k_te_cg    -- the structural rank-one terms and the CG update (one CTA).
// FP64 issues at a low rate on this part, so the point work is spread over 16 lanes per point and over
// several CTAs, and reductions are combined by one warp.
// The FSI and CG loops run on the device as CUDA-graph WHILE nodes whose conditions the kernels set (a step
// needs no host round trip); eager steps read the same flags on the host after each iteration.  Every loop is
// bounded by an iteration counter that the kernel setting its condition increments.
#include <cmath>
#include "internal.h"

namespace {

constexpr int kThr = 256;            // one-CTA kernels (CG update, FSI update, step end)
constexpr int kPtThr = 128;          // point kernels: 16 lanes per point, 8 points per CTA
constexpr int kPtCta = kPtThr / 16;
constexpr int kMaxB = 64;            // bodies per context
constexpr int kSrcChunk = 64;        // selected points whose face contributions one source CTA stages at a time
constexpr unsigned FULL = 0xffffffffu;

using TePoint = FaceWindow;  // the 4 x 4 face windows of one body point (internal.h)

// control words
enum { TC_CG_IT = 0, TC_CG_DONE, TC_FSI_IT, TC_FSI_DONE, TC_CG_STEP, TC_CG_LAST, TC_N };
// scalars: r.r and the stopping threshold on r.r
enum { TS_RR = 0, TS_THR, TS_N };

struct TeArgs {
  const void* s0;  // level-0 streamfunction after the predictor (s*), context precision
  const void* ts;  // level-0 streamfunction of the operator application
  int fp64;
  long ps;
  double x0, y0, h, inv_h, dt, ds, U, V, tol, ktol, two_dt, four_dt2;
  double kscale_h;  // ds / h^3: (ds / h^2) E C with the 1/h of C
  int max_iters, kmax;
  int nb, nf, n_bodies;
  int i_lo, i_hi, j_lo, j_hi;  // Omega_0 vertex box: every body point must lie inside
  const BodyDev* bodies;
  BodyState* st;
  const int* point_body;
  const double* rpts;
  const double* rur;
  TePoint* pt;
  double *f, *r, *p, *q, *rhs, *sv;
  double* scal;
  int* ctl;
  unsigned long long* cg_total;
  int* status;
  int* ctrl;
  double* hist;
  int hist_cap;
  cudaGraphConditionalHandle h_fsi, h_cg;
  int use_cond;
  const double* kin;  // prescribed kinematics [kin_cap][n_bodies][6] or NULL
  int kin_cap;
};

__device__ __forceinline__ double load_s(const void* s, int fp64, long o) {
  return fp64 ? ((const double*)s)[o] : (double)((const float*)s)[o];
}

// deterministic block sum, result in every thread (red: 33 doubles).  FP64 issues at a low rate on this
// part, so the partials are combined by one warp, not by every thread.
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();  // red may still be read after a previous call
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__device__ __forceinline__ double group16_sum(double v) {
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o, 16);
  return v;
}

// ---------------------------------------------------------------------------------------------------------
// Start of an FSI iteration (8 points per CTA, 16 lanes per point): body points of the iterate, their face
// windows and delta weights (one weight per lane), S, and the right-hand side
//   r^c(k) = E (C s* + q_inf) - u_rigid - S phi^(k) + S (r^theta(k) - (2/dt) r^phi(k) / J).
// Every CTA derives the structural terms of the step from the body state; CTA 0 stores them and starts the
// CG solve from the current f.
__global__ void __launch_bounds__(kPtThr) k_te_prep(TeArgs a) {
  __shared__ double b_th[kMaxB], b_ph[kMaxB], b_jac[kMaxB], b_rphi[kMaxB], b_rth[kMaxB], b_sn[kMaxB], b_cs[kMaxB];
  // moving hinges and driven plates (Sec. 5.1): reference point or hinge, its velocity, alpha1', and for a
  // driven plate its direction (sin, -cos)(alpha1)
  __shared__ double b_hx[kMaxB], b_hy[kMaxB], b_vx[kMaxB], b_vy[kMaxB], b_ad[kMaxB], b_sa[kMaxB], b_ca[kMaxB];
  const int tid = threadIdx.x, nb = a.nb;
  const bool first = a.ctl[TC_FSI_IT] == 0;
  for (int bi = tid; bi < a.n_bodies; bi += kPtThr) {
    const BodyDev b = a.bodies[bi];
    const BodyState s = a.st[bi];
    double jac = 1.0, rphi = 0.0, rth = 0.0, th = 0.0, ph = 0.0, t0 = b.theta0, g = 0.0;
    b_hx[bi] = b.hx;
    b_hy[bi] = b.hy;
    b_vx[bi] = b_vy[bi] = b_ad[bi] = b_sa[bi] = b_ca[bi] = 0.0;
    const int src = b.type == FSI_BODY_DRIVEN ? bi : (b.type == FSI_BODY_TORSIONAL ? b.driver : -1);
    const double* q = (a.kin && src >= 0) ? a.kin + ((long)(a.ctrl[2] % a.kin_cap) * a.n_bodies + src) * 6 : nullptr;
    if (b.type == FSI_BODY_TORSIONAL) {
      const double dt = a.dt;
      jac = 4.0 * b.inertia / (dt * dt) + 2.0 * b.damping / dt + b.stiffness;
      rphi = b.inertia * (4.0 * s.theta / (dt * dt) + 4.0 * s.phi / dt + s.phidot) +
             b.damping * (2.0 * s.theta / dt + s.phi);
      rth = s.phi + 2.0 / dt * s.theta;
      th = first ? s.theta : s.theta_k;
      ph = first ? s.phi : s.phi_k;
    }
    if (q) {
      double sa, ca;
      sincos(q[3], &sa, &ca);
      if (b.type == FSI_BODY_DRIVEN) {
        b_hx[bi] = b.hx + q[0];
        b_vx[bi] = q[1];
        b_sa[bi] = sa;
        b_ca[bi] = ca;
        b_ad[bi] = q[4];
      } else {  // hinge at l1 along the driven plate; g of Eq. newtonseldg at the iterate
        const BodyDev d = a.bodies[src];
        b_hx[bi] = d.hx + q[0] + b.l1 * sa;
        b_hy[bi] = d.hy - b.l1 * ca;
        b_vx[bi] = q[1] + b.l1 * q[4] * ca;
        b_vy[bi] = b.l1 * q[4] * sa;
        b_ad[bi] = q[4];
        t0 = q[3] - 0.5 * M_PI;
        const double ml = b.mass * b.l1 * b.l2;
        g = -b.mass * b.l2 * cos(q[3] + th) * q[2] - (b.inertia + ml * cos(th)) * q[5] - ml * sin(th) * q[4] * q[4];
      }
    }
    b_th[bi] = th;
    b_ph[bi] = ph;
    b_jac[bi] = jac;
    b_rphi[bi] = rphi + g;
    b_rth[bi] = rth;
    sincos(t0 + th, &b_sn[bi], &b_cs[bi]);
    if (blockIdx.x == 0) {
      BodyState& w = a.st[bi];
      w.gk = g;
      w.t0 = t0;
      if (first) {
        w.jac = jac;
        w.kc = (2.0 * a.ds / a.dt) / jac;
        w.r_phi = rphi;
        w.r_theta = rth;
        w.theta_k = s.theta;
        w.phi_k = s.phi;
        w.theta_p = s.theta;
      }
    }
  }
  __syncthreads();
  const int l = tid & 15, d = l & 3, e = l >> 2;
  const int p = blockIdx.x * kPtCta + (tid >> 4);
  const bool act = p < nb;
  const int pp = act ? p : nb - 1;
  const int bi = a.point_body[pp];
  const BodyDev b = a.bodies[bi];
  double x, y, svx = 0.0, svy = 0.0, ux = 0.0, uy = 0.0;
  if (b.type == FSI_BODY_TORSIONAL) {
    const double sn = b_sn[bi], cs = b_cs[bi];
    const double q = (double)(pp - b.off) * a.ds;
    x = __dadd_rn(b_hx[bi], __dmul_rn(q, cs));
    y = __dadd_rn(b_hy[bi], __dmul_rn(q, sn));
    svx = q * (-sn);
    svy = q * cs;
    const double th_k = b_th[bi], ph_k = b_ph[bi];
    const double rphik = b_rphi[bi] - b_jac[bi] * th_k;
    const double rthk = b_rth[bi] - a.two_dt * th_k + ph_k;
    const double coef = rthk - a.two_dt * rphik / b_jac[bi];
    // moving hinge: its velocity and alpha1' q R are known parts of the point velocities
    ux = svx * ph_k - svx * coef + b_vx[bi] + b_ad[bi] * svx;
    uy = svy * ph_k - svy * coef + b_vy[bi] + b_ad[bi] * svy;
  } else if (b.type == FSI_BODY_DRIVEN) {  // prescribed heave and pitch
    const double sj = b.s_lo + (double)(pp - b.off) * a.ds;
    x = b_hx[bi] + sj * b_sa[bi];
    y = b_hy[bi] - sj * b_ca[bi];
    ux = b_vx[bi] + sj * b_ad[bi] * b_ca[bi];
    uy = sj * b_ad[bi] * b_sa[bi];
  } else {
    x = a.rpts[2 * pp];
    y = a.rpts[2 * pp + 1];
    ux = a.rur[2 * pp];
    uy = a.rur[2 * pp + 1];
  }
  double X = (x - a.x0) / a.h, Y = (y - a.y0) / a.h;
  if (!(X >= (double)a.i_lo && X <= (double)a.i_hi && Y >= (double)a.j_lo && Y <= (double)a.j_hi)) {
    if (act && l == 0) dev_set_status(a.status, FSI_ERR_BODY_OUTSIDE_SUBDOMAIN);
    X = fmin(fmax(isfinite(X) ? X : (double)a.i_lo, (double)a.i_lo), (double)a.i_hi);
    Y = fmin(fmax(isfinite(Y) ? Y : (double)a.j_lo, (double)a.j_lo), (double)a.j_hi);
  }
  // windows: u faces offset (0, 1/2) from the vertices, v faces (1/2, 0)
  const int iu = (int)floor(X) - 1, ju = (int)floor(Y - 0.5) - 1;
  const int iv = (int)floor(X - 0.5) - 1, jv = (int)floor(Y) - 1;
  // lane l evaluates weight l: 0-3 x of u, 4-7 y of u, 8-11 x of v, 12-15 y of v
  const int k = l & 3, which = l >> 2;
  double r;
  if (which == 0) r = __dsub_rn((double)(iu + k), X);
  else if (which == 1) r = __dsub_rn(__dadd_rn((double)(ju + k), 0.5), Y);
  else if (which == 2) r = __dsub_rn(__dadd_rn((double)(iv + k), 0.5), X);
  else r = __dsub_rn((double)(jv + k), Y);
  const double wl = delta3_rn(r);
  const double wxu = __shfl_sync(FULL, wl, d, 16), wyu = __shfl_sync(FULL, wl, 4 + e, 16);
  const double wxv = __shfl_sync(FULL, wl, 8 + d, 16), wyv = __shfl_sync(FULL, wl, 12 + e, 16);
  // face (d, e) terms of E (C s* + q_inf): u = (s[J+1][I] - s[J][I]) / h + U, v = -(s[J][I+1] - s[J][I]) / h + V
  const long Iu = iu + d, Ju = ju + e, Iv = iv + d, Jv = jv + e;
  const double du = load_s(a.s0, a.fp64, (Ju + 1) * a.ps + Iu) - load_s(a.s0, a.fp64, Ju * a.ps + Iu);
  const double dv = load_s(a.s0, a.fp64, Jv * a.ps + Iv + 1) - load_s(a.s0, a.fp64, Jv * a.ps + Iv);
  const double eu = group16_sum(__dmul_rn(__dmul_rn(wxu, wyu), du * a.inv_h + a.U));
  const double ev = group16_sum(__dmul_rn(__dmul_rn(wxv, wyv), -dv * a.inv_h + a.V));
  if (act) {
    TePoint* P = a.pt + p;
    P->w[l] = wl;
    if (l == 0) {
      P->iu = iu;
      P->ju = ju;
      P->iv = iv;
      P->jv = jv;
      a.rhs[p] = eu - ux;
      a.rhs[nb + p] = ev - uy;
      a.sv[p] = svx;
      a.sv[nb + p] = svy;
    }
  }
  if (blockIdx.x == 0) {
    for (int m = tid; m < a.nf; m += kPtThr) a.p[m] = a.f[m];  // the first application is K f (CG start)
    if (tid == 0) {
      a.ctl[TC_CG_IT] = 0;
      a.ctl[TC_CG_DONE] = 0;
      if (a.use_cond) cudaGraphSetConditional(a.h_cg, 1u);
    }
  }
}

// curl of E^T v (scaled by pre_h = pre / h) at the interior vertices of the box [wi0, wi1] x [wj0, wj1]:
// src(i, j) = pre ((Fv(i+1/2, j) - Fv(i-1/2, j)) - (Fu(i, j+1/2) - Fu(i, j-1/2))) / h, the face values F summing
// (weight * v) over the points in point order.  A CTA takes a 32 x 4 tile: it selects (in point order) the
// points whose faces enter its curls, stages their 32 face contributions in chunks, and each thread sums
// those of its vertex.
template <typename T>
__global__ void __launch_bounds__(128) k_te_src(T* __restrict__ src, long ps, int wi0, int wi1, int wj0, int wj1,
                                                const TePoint* __restrict__ pt, const double* __restrict__ vec,
                                                int nb, double pre_h) {
  extern __shared__ __align__(16) unsigned char te_smem[];
  double* sc = reinterpret_cast<double*>(te_smem);          // [kSrcChunk][32] face contributions
  int* si = reinterpret_cast<int*>(sc + kSrcChunk * 32);    // [nb][4] windows of the selected points
  int* sp = si + 4 * nb;                                     // [nb] their point indices
  __shared__ int wcount[4], n_sel;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ti0 = wi0 + (int)blockIdx.x * 32, tj0 = wj0 + (int)blockIdx.y * 4;
  if (tid == 0) n_sel = 0;
  __syncthreads();
  // a point's faces enter the curls at vertices i in [iu - 1, iu + 4], j in [ju - 1, ju + 4] (superset)
  for (int base = 0; base < nb; base += 128) {
    const int p = base + tid;
    int iu = 0, ju = 0;
    bool take = false;
    if (p < nb) {
      iu = pt[p].iu;
      ju = pt[p].ju;
      take = iu - 1 <= ti0 + 31 && iu + 4 >= ti0 && ju - 1 <= tj0 + 3 && ju + 4 >= tj0;
    }
    const unsigned m = __ballot_sync(FULL, take);
    if (lane == 0) wcount[wid] = __popc(m);
    __syncthreads();
    int off = n_sel;
    for (int w = 0; w < wid; ++w) off += wcount[w];
    if (take) {
      const int q = off + __popc(m & ((1u << lane) - 1u));
      si[4 * q] = iu;
      si[4 * q + 1] = ju;
      si[4 * q + 2] = pt[p].iv;
      si[4 * q + 3] = pt[p].jv;
      sp[q] = p;
    }
    __syncthreads();
    if (tid == 0) n_sel += wcount[0] + wcount[1] + wcount[2] + wcount[3];
    __syncthreads();
  }
  const int ns = n_sel;
  const int i = ti0 + lane, j = tj0 + wid;
  double fun = 0.0, fus = 0.0, fve = 0.0, fvw = 0.0;
  for (int c0 = 0; c0 < ns; c0 += kSrcChunk) {
    const int nc = ns - c0 < kSrcChunk ? ns - c0 : kSrcChunk;
    __syncthreads();  // the previous chunk's contributions have been read
    for (int t = tid; t < 16 * nc; t += 128) {
      const int qq = t >> 4, l = t & 15, d = l & 3, e = l >> 2;
      const int p = sp[c0 + qq];
      const double* w = pt[p].w;
      sc[32 * qq + l] = __dmul_rn(__dmul_rn(w[d], w[4 + e]), vec[p]);             // u face (iu + d, ju + e)
      sc[32 * qq + 16 + l] = __dmul_rn(__dmul_rn(w[8 + d], w[12 + e]), vec[nb + p]);  // v face (iv + d, jv + e)
    }
    __syncthreads();
    for (int qq = 0; qq < nc; ++qq) {
      const int* wv = si + 4 * (c0 + qq);
      const double* cq = sc + 32 * qq;
      const int du = i - wv[0];
      if ((unsigned)du < 4u) {
        const int en = j - wv[1], es = j - 1 - wv[1];
        if ((unsigned)en < 4u) fun += cq[en * 4 + du];
        if ((unsigned)es < 4u) fus += cq[es * 4 + du];
      }
      const int ev = j - wv[3];
      if ((unsigned)ev < 4u) {
        const int de = i - wv[2], dw = i - 1 - wv[2];
        if ((unsigned)de < 4u) fve += cq[16 + ev * 4 + de];
        if ((unsigned)dw < 4u) fvw += cq[16 + ev * 4 + dw];
      }
    }
  }
  if (i <= wi1 && j <= wj1) src[(long)(j - 1) * ps + (i - 1)] = T(pre_h * ((fve - fvw) - (fun - fus)));
}

// E C s_t at the body points (8 points per CTA, 16 lanes per point): q = (ds / h^3) sum w (s differences).
__global__ void __launch_bounds__(kPtThr) k_te_apply(TeArgs a) {
  const int tid = threadIdx.x, nb = a.nb, l = tid & 15, d = l & 3, e = l >> 2;
  const int p = blockIdx.x * kPtCta + (tid >> 4);
  const int pp = p < nb ? p : nb - 1;
  const TePoint* P = a.pt + pp;
  const long Iu = P->iu + d, Ju = P->ju + e, Iv = P->iv + d, Jv = P->jv + e;
  const double du = load_s(a.ts, a.fp64, (Ju + 1) * a.ps + Iu) - load_s(a.ts, a.fp64, Ju * a.ps + Iu);
  const double dv = load_s(a.ts, a.fp64, Jv * a.ps + Iv + 1) - load_s(a.ts, a.fp64, Jv * a.ps + Iv);
  const double qu = group16_sum((P->w[d] * P->w[4 + e]) * du);
  const double qv = group16_sum(-(P->w[8 + d] * P->w[12 + e]) * dv);
  if (p < nb && l == 0) {
    a.q[p] = a.kscale_h * qu;
    a.q[nb + p] = a.kscale_h * qv;
  }
}

// One CG iteration after the operator application: q += sum_b kc_b S_b (S_b . p) (the structural rank-one
// terms, kc = (2 ds/dt)/J), then (iteration 0) r = rhs - q, p = r, or (later) the CG update of f, r and p.
// Sets the CG loop condition on every path.
__global__ void __launch_bounds__(kThr) k_te_cg(TeArgs a) {
  __shared__ double red[33];
  __shared__ double s_div;
  const int tid = threadIdx.x, nb = a.nb, nf = a.nf;
  const int it = a.ctl[TC_CG_IT];
  for (int bi = 0; bi < a.n_bodies; ++bi) {
    const BodyDev b = a.bodies[bi];
    if (b.type != FSI_BODY_TORSIONAL) continue;
    double part = 0.0;
    for (int m = b.off + tid; m < b.off + b.n; m += kThr) part += a.sv[m] * a.p[m] + a.sv[nb + m] * a.p[nb + m];
    const double dot = block_sum(part, red) * a.st[bi].kc;
    for (int m = b.off + tid; m < b.off + b.n; m += kThr) {
      a.q[m] += a.sv[m] * dot;
      a.q[nb + m] += a.sv[nb + m] * dot;
    }
  }
  __syncthreads();
  bool done;
  if (it == 0) {
    double prr = 0.0, pbb = 0.0;
    for (int m = tid; m < nf; m += kThr) {
      const double rk = a.rhs[m] - a.q[m];
      a.r[m] = rk;
      a.p[m] = rk;
      prr += rk * rk;
      pbb += a.rhs[m] * a.rhs[m];
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
    for (int m = tid; m < nf; m += kThr) ppq += a.p[m] * a.q[m];
    const double pq = block_sum(ppq, red);
    const double rr = a.scal[TS_RR];
    if (tid == 0) s_div = rr / pq;
    __syncthreads();
    const double alpha = s_div;
    double prr = 0.0;
    for (int m = tid; m < nf; m += kThr) {
      a.f[m] += alpha * a.p[m];
      const double rk = a.r[m] - alpha * a.q[m];
      a.r[m] = rk;
      prr += rk * rk;
    }
    const double rn = block_sum(prr, red);
    if (tid == 0) s_div = rn / rr;
    __syncthreads();
    const double beta = s_div;
    for (int m = tid; m < nf; m += kThr) a.p[m] = a.r[m] + beta * a.p[m];
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
  __shared__ double red[33];
  const int tid = threadIdx.x, nb = a.nb;
  double dmax = 0.0;
  bool finite = true;
  for (int bi = 0; bi < a.n_bodies; ++bi) {
    const BodyDev b = a.bodies[bi];
    if (b.type != FSI_BODY_TORSIONAL) continue;
    double part = 0.0;
    for (int m = b.off + tid; m < b.off + b.n; m += kThr) part += a.sv[m] * a.f[m] + a.sv[nb + m] * a.f[nb + m];
    const double sf = block_sum(part, red);
    BodyState& s = a.st[bi];
    const double dth = (s.r_phi + s.gk - s.jac * s.theta_k + a.ds * sf) / s.jac;
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
  __shared__ double red[33];
  const int tid = threadIdx.x, nb = a.nb;
  const int slot = a.ctrl[2] % a.hist_cap;
  const int iters = a.ctl[TC_FSI_IT];
  for (int bi = 0; bi < a.n_bodies; ++bi) {
    const BodyDev b = a.bodies[bi];
    double sn = 0.0, cs = 0.0;
    if (b.type == FSI_BODY_TORSIONAL) sincos(a.st[bi].t0 + a.st[bi].theta_p, &sn, &cs);
    double px = 0.0, py = 0.0, pm = 0.0;
    for (int m = b.off + tid; m < b.off + b.n; m += kThr) {
      const double fxp = a.f[m], fyp = a.f[nb + m];
      const double q = (double)(m - b.off) * a.ds;
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
  a.inv_h = 1.0 / c->g.h;
  a.dt = c->g.dt;
  a.ds = c->ds;
  a.U = c->g.uinf[0];
  a.V = c->g.uinf[1];
  a.tol = c->x.tol;
  a.ktol = c->x.krylov_tol;
  a.two_dt = 2.0 / c->g.dt;
  a.four_dt2 = 4.0 / (c->g.dt * c->g.dt);
  a.kscale_h = c->ds / (c->g.h * c->g.h * c->g.h);
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
  a.q = c->d_te_q;
  a.rhs = c->d_rhs;
  a.sv = c->d_sv;
  a.scal = c->d_te_scal;
  a.ctl = c->d_te_ctl;
  a.cg_total = c->d_te_total;
  a.status = c->d_status;
  a.ctrl = c->d_ctrl;
  a.hist = c->d_hist;
  a.hist_cap = c->hist_cap;
  a.kin = c->d_kin;
  a.kin_cap = c->kin_cap > 0 ? c->kin_cap : 1;
  return a;
}

size_t src_smem(int nb) { return (size_t)kSrcChunk * 32 * sizeof(double) + (size_t)nb * 5 * sizeof(int); }

// curl of E^T vec (times pre) into the source buffer; the vertex box is the interior part of Omega_0 grown by
// 3 cells, which holds the support of every point inside Omega_0
template <typename T>
fsi_status launch_src(fsi_ctx* c, const double* vec, double pre) {
  const int wi0 = c->i_lo - 3 < 1 ? 1 : c->i_lo - 3, wi1 = c->i_hi + 3 > c->nx - 1 ? c->nx - 1 : c->i_hi + 3;
  const int wj0 = c->j_lo - 3 < 1 ? 1 : c->j_lo - 3, wj1 = c->j_hi + 3 > c->ny - 1 ? c->ny - 1 : c->j_hi + 3;
  const dim3 grid((wi1 - wi0 + 32) / 32, (wj1 - wj0 + 4) / 4);
  FSI_CUDA_TRY(raise_smem_limit(k_te_src<T>, src_smem(c->nb)));
  k_te_src<T><<<grid, 128, src_smem(c->nb), c->stream>>>((T*)c->src, c->ps, wi0, wi1, wj0, wj1,
                                                           (const TePoint*)c->d_te_pt, vec, c->nb, pre / c->g.h);
  FSI_CUDA_TRY(cudaGetLastError());
  c->launches_per_step += 1;
  return FSI_OK;
}

fsi_status launch_src_any(fsi_ctx* c, const double* vec, double pre) {
  return c->prec == FSI_PREC_FP64 ? launch_src<double>(c, vec, pre) : launch_src<float>(c, vec, pre);
}

fsi_status launch_one(fsi_ctx* c, void (*k)(TeArgs), const TeArgs& a) {
  k<<<1, kThr, 0, c->stream>>>(a);
  FSI_CUDA_TRY(cudaGetLastError());
  c->launches_per_step += 1;
  return FSI_OK;
}

fsi_status launch_points(fsi_ctx* c, void (*k)(TeArgs), const TeArgs& a) {
  k<<<(c->nb + kPtCta - 1) / kPtCta, kPtThr, 0, c->stream>>>(a);
  FSI_CUDA_TRY(cudaGetLastError());
  c->launches_per_step += 1;
  return FSI_OK;
}

// one CG iteration: operator application to p (source, the three passes, interpolation), then the update
fsi_status cg_iteration(fsi_ctx* c, const TeArgs& a) {
  fsi_status st = launch_src_any(c, c->d_te_p, 1.0);
  if (st != FSI_OK) return st;
  st = launch_level_solve(c, 0, c->src, c->te_w, c->te_s, 0, 0);
  if (st != FSI_OK) return st;
  st = launch_points(c, k_te_apply, a);
  if (st != FSI_OK) return st;
  return launch_one(c, k_te_cg, a);
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
    fsi_status st = launch_points(c, k_te_prep, a);
    if (st != FSI_OK) return st;
    for (int k = 0; k < c->x.krylov_max_iters; ++k) {
      st = cg_iteration(c, a);
      if (st != FSI_OK) return st;
      int done = 0;
      st = read_flag(c, TC_CG_DONE, &done);
      if (st != FSI_OK) return st;
      if (done) break;
    }
    st = launch_one(c, k_te_post, a);
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
    s = launch_points(c, k_te_prep, a);
    if (s != FSI_OK) return s;
    s = capture_while(c, c->te_stream[1], a.h_cg, [&]() -> fsi_status { return cg_iteration(c, a); });
    if (s != FSI_OK) return s;
    return launch_one(c, k_te_post, a);
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
  return launch_one(c, k_te_finish, a);
}

// kernel attributes (dynamic shared memory of the source kernel for nb points)
fsi_status true_e_setup(fsi_ctx* c) {
  const int sm = (int)src_smem(c->nb);
  FSI_CUDA_TRY(raise_smem_limit(k_te_src<double>, (size_t)sm));
  FSI_CUDA_TRY(raise_smem_limit(k_te_src<float>, (size_t)sm));
  return FSI_OK;
}

size_t true_e_point_bytes() { return sizeof(TePoint); }
