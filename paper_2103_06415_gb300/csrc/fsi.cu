// FSI iteration of one time step (Algorithm 2; Eqs. stress2 and dtheta2) in double precision, as one
// cooperative kernel over a fixed set of CTAs:
//   A  body points at theta^(k), the hat map P (Eq. weights), rhs = P E0 (C s* + q_inf) - r^c(k)
//      + S^T (r^theta(k) - (2/dt) J^{-1} r^phidot(k))                                   [all CTAs]
//   B  K = (ds/h^2) P B0 P^T + (2 ds/dt) S^T J^{-1} S  (16 B0 lookups per entry)          [all CTAs]
//   C  f = K^{-1} rhs to double accuracy: blocked Cholesky of K rounded to float in the shared memory of
//      CTA 0, three solves with that factor separated by double residuals r = rhs - K f   [CTA 0 + all]
//   D  dtheta = J^{-1}(r^phidot(k) + ds S f), convergence on max |dtheta|                 [CTA 0]
// repeated until max |dtheta| <= tol, then the Newmark update and force outputs.
// Data written by other CTAs inside this kernel is read with __ldcg (L2), so no stale L1 line is used.
#include <cooperative_groups.h>
#include <cmath>
#include "internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr int kSolves = 3;  // factor solves; kSolves-1 double residuals in between
constexpr int BS = 32;      // Cholesky block (one warp)
constexpr unsigned FULL = 0xffffffffu;

struct FsiArgs {
  const void* s0;
  int fp64;
  long ps;
  double x0, y0, h, dt, ds, U, V, tol;
  int max_iters;
  int n_sd, ni, nj, i_lo, j_lo;
  const double* B0;
  int nb, nf, n_bodies;
  const BodyDev* bodies;
  BodyState* st;
  const int* point_body;
  const double* rpts;
  const double* rur;
  int* pidx;
  double* pw;
  double* sv;
  double* rhs;  // [nf] right-hand side, then [nf] residual
  double* K;
  double* f;
  int* ctrl;
  int* status;
  double* hist;
  int hist_cap;
};

__device__ __forceinline__ double load_s(const FsiArgs& a, long o) {
  return a.fp64 ? ((const double*)a.s0)[o] : (double)((const float*)a.s0)[o];
}

// E0 (C s + q_inf) at level-0 vertex (I, J): u = sum_d w_d (s[J+1][I+d] - s[J-1][I+d])/(2h) + U,
// v = -sum_d w_d (s[J+d][I+1] - s[J+d][I-1])/(2h) + V with w = (1/6, 2/3, 1/6).
__device__ void e0cs(const FsiArgs& a, int I, int J, double* u, double* v) {
  const double w[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
  double su = 0.0, sv = 0.0;
  for (int d = -1; d <= 1; ++d) {
    su += w[d + 1] * (load_s(a, (long)(J + 1) * a.ps + I + d) - load_s(a, (long)(J - 1) * a.ps + I + d));
    sv += w[d + 1] * (load_s(a, (long)(J + d) * a.ps + I + 1) - load_s(a, (long)(J + d) * a.ps + I - 1));
  }
  *u = su / (2.0 * a.h) + a.U;
  *v = -sv / (2.0 * a.h) + a.V;
}

// Deterministic block sum (fixed tree); all threads must call; result valid in every thread.
__device__ double block_sum(double x, double* red) {
  const int tid = threadIdx.x;
  red[tid] = x;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Blocked right-looking Cholesky of the lower triangle of L (row stride ld) in shared memory.
// Returns false (in every thread) if a pivot is not positive.
__device__ bool chol_blocked(float* L, int n, int ld, int* bad) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) *bad = 0;
  __syncthreads();
  for (int jb = 0; jb < n; jb += BS) {
    const int bs = min(BS, n - jb);
    if (wid == 0) {  // diagonal block in registers: lane r holds row jb + r
      float a[BS];
#pragma unroll
      for (int c = 0; c < BS; ++c) a[c] = (lane < bs && c < bs) ? L[(long)(jb + lane) * ld + jb + c] : 0.0f;
#pragma unroll
      for (int c = 0; c < BS; ++c)
        if (lane >= bs && c == lane) a[c] = 1.0f;  // identity padding keeps the padded factor defined
#pragma unroll
      for (int c = 0; c < BS; ++c) {
        float d = __shfl_sync(FULL, a[c], c);
        if (!(d > 0.0f)) {
          if (lane == 0 && c < bs) *bad = 1;
          d = 1.0f;
        }
        d = sqrtf(d);
        if (lane == c) a[c] = d;
        if (lane > c) a[c] /= d;
#pragma unroll
        for (int cc = c + 1; cc < BS; ++cc) {
          const float lcc = __shfl_sync(FULL, a[c], cc);
          if (lane > c && cc <= lane) a[cc] -= a[c] * lcc;
        }
      }
      if (lane < bs) {
#pragma unroll
        for (int c = 0; c < BS; ++c)
          if (c <= lane && c < bs) L[(long)(jb + lane) * ld + jb + c] = a[c];
      }
    }
    __syncthreads();
    // panel: rows below solve X Ldiag^T = A (row-wise forward substitution)
    for (int i = jb + bs + tid; i < n; i += blockDim.x) {
      float* row = L + (long)i * ld + jb;
      for (int c = 0; c < bs; ++c) {
        float v = row[c];
        const float* dr = L + (long)(jb + c) * ld + jb;
        for (int cc = 0; cc < c; ++cc) v -= row[cc] * dr[cc];
        row[c] = v / dr[c];
      }
    }
    __syncthreads();
    // trailing update A22 -= L21 L21^T (lower part), one warp per row
    const int t0 = jb + bs;
    for (int i = t0 + wid; i < n; i += nw) {
      const float* ri = L + (long)i * ld + jb;
      for (int k = t0 + lane; k <= i; k += 32) {
        const float* rk = L + (long)k * ld + jb;
        float acc = 0.0f;
        for (int c = 0; c < bs; ++c) acc += ri[c] * rk[c];
        L[(long)i * ld + k] -= acc;
      }
    }
    __syncthreads();
  }
  return *bad == 0;
}

// y <- (L L^T)^{-1} y with the blocked factor (float, in shared memory).
__device__ void chol_solve(const float* L, int n, int ld, float* y) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nblk = (n + BS - 1) / BS;
  for (int b = 0; b < nblk; ++b) {  // forward
    const int jb = b * BS, bs = min(BS, n - jb);
    if (wid == 0) {
      float v = lane < bs ? y[jb + lane] : 0.0f;
      for (int c = 0; c < bs; ++c) {
        const float yc = __shfl_sync(FULL, v, c) / L[(long)(jb + c) * ld + jb + c];
        if (lane == c) v = yc;
        if (lane > c && lane < bs) v -= L[(long)(jb + lane) * ld + jb + c] * yc;
      }
      if (lane < bs) y[jb + lane] = v;
    }
    __syncthreads();
    for (int i = jb + bs + tid; i < n; i += blockDim.x) {
      const float* ri = L + (long)i * ld + jb;
      float acc = 0.0f;
      for (int c = 0; c < bs; ++c) acc += ri[c] * y[jb + c];
      y[i] -= acc;
    }
    __syncthreads();
  }
  for (int b = nblk - 1; b >= 0; --b) {  // backward with L^T
    const int jb = b * BS, bs = min(BS, n - jb);
    if (wid == 0) {
      float v = lane < bs ? y[jb + lane] : 0.0f;
      for (int c = bs - 1; c >= 0; --c) {
        const float xc = __shfl_sync(FULL, v, c) / L[(long)(jb + c) * ld + jb + c];
        if (lane == c) v = xc;
        if (lane < c) v -= L[(long)(jb + c) * ld + jb + lane] * xc;
      }
      if (lane < bs) y[jb + lane] = v;
    }
    __syncthreads();
    for (int i = tid; i < jb; i += blockDim.x) {
      float acc = 0.0f;
      for (int c = 0; c < bs; ++c) acc += L[(long)(jb + c) * ld + i] * y[jb + c];
      y[i] -= acc;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_fsi(FsiArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ double red[256];
  __shared__ int sh_flag, sh_bad;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const long gtid = (long)blockIdx.x * nthr + tid;
  const long gsize = (long)gridDim.x * nthr;
  const int nb = a.nb, nf = a.nf;
  const int ld = nf | 1;
  const double dt = a.dt;
  double* res = a.rhs + nf;

  if (blockIdx.x == 0 && tid < a.n_bodies) {
    const BodyDev b = a.bodies[tid];
    BodyState& s = a.st[tid];
    if (b.type == FSI_BODY_TORSIONAL) {
      s.jac = 4.0 * b.inertia / (dt * dt) + 2.0 * b.damping / dt + b.stiffness;
      s.r_phi = b.inertia * (4.0 * s.theta / (dt * dt) + 4.0 * s.phi / dt + s.phidot) +
                b.damping * (2.0 * s.theta / dt + s.phi);
      s.r_theta = s.phi + 2.0 / dt * s.theta;
      s.theta_k = s.theta;
      s.phi_k = s.phi;
    }
  }
  if (gtid == 0) a.ctrl[0] = 0;
  if (tid == 0) sh_flag = 0;
  grid.sync();

  int it = 0;
  for (; it < a.max_iters; ++it) {
    // ---- A: body points, P, right-hand side
    for (long p = gtid; p < nb; p += gsize) {
      const int bi = a.point_body[p];
      const BodyDev b = a.bodies[bi];
      const double th_k = __ldcg(&a.st[bi].theta_k), ph_k = __ldcg(&a.st[bi].phi_k);
      const double s_rphi = __ldcg(&a.st[bi].r_phi), s_rth = __ldcg(&a.st[bi].r_theta);
      const double s_jac = __ldcg(&a.st[bi].jac);
      double x, y, svx = 0.0, svy = 0.0, ucx, ucy, coef = 0.0;
      if (b.type == FSI_BODY_TORSIONAL) {
        const int j = (int)p - b.off;
        const double ang = b.theta0 + th_k;
        double sn, cs;
        sincos(ang, &sn, &cs);
        x = b.hx + (double)j * a.ds * cs;
        y = b.hy + (double)j * a.ds * sn;
        svx = (double)j * a.ds * (-sn);
        svy = (double)j * a.ds * cs;
        ucx = svx * ph_k;
        ucy = svy * ph_k;
        const double rphik = s_rphi - s_jac * th_k;
        const double rthk = s_rth - 2.0 / dt * th_k + ph_k;
        coef = rthk - 2.0 / dt * rphik / s_jac;
      } else {
        x = a.rpts[2 * p];
        y = a.rpts[2 * p + 1];
        ucx = a.rur[2 * p];
        ucy = a.rur[2 * p + 1];
      }
      const double xl = a.x0 + a.i_lo * a.h, yl = a.y0 + a.j_lo * a.h;
      const double fx = (x - xl) / a.h, fy = (y - yl) / a.h;
      int ci = (int)floor(fx), cj = (int)floor(fy);
      if (!(fx >= 0.0 && fy >= 0.0 && fx <= (double)(a.ni - 1) && fy <= (double)(a.nj - 1))) {
        dev_set_status(a.status, FSI_ERR_BODY_OUTSIDE_SUBDOMAIN);
        ci = 0;
        cj = 0;
      }
      ci = min(max(ci, 0), a.ni - 2);
      cj = min(max(cj, 0), a.nj - 2);
      const double rx = fx - ci, ry = fy - cj;
      const double wts[4] = {(1.0 - rx) * (1.0 - ry), rx * (1.0 - ry), (1.0 - rx) * ry, rx * ry};
      double ubx = 0.0, uby = 0.0;
      for (int q = 0; q < 4; ++q) {
        const int aa = q & 1, bb = q >> 1;
        a.pidx[4 * p + q] = (cj + bb) * a.ni + (ci + aa);
        a.pw[4 * p + q] = wts[q];
        double u, v;
        e0cs(a, a.i_lo + ci + aa, a.j_lo + cj + bb, &u, &v);
        ubx += wts[q] * u;
        uby += wts[q] * v;
      }
      a.sv[2 * p] = svx;
      a.sv[2 * p + 1] = svy;
      a.rhs[p] = ubx - ucx + svx * coef;
      a.rhs[nb + p] = uby - ucy + svy * coef;
    }
    grid.sync();
    // ---- B: K = (ds/h^2) P B0 P^T + (2 ds/dt) S^T J^{-1} S (both triangles written)
    const double kscale = a.ds / (a.h * a.h);
    const long n2 = 2L * a.n_sd;
    for (long e = gtid; e < (long)nf * nf; e += gsize) {
      const int r = (int)(e / nf), cidx = (int)(e % nf);
      if (cidx > r) continue;
      const int ca = r / nb, pa = r % nb, cb = cidx / nb, pb = cidx % nb;
      double acc = 0.0;
      int ib[4];
      double wb[4];
#pragma unroll
      for (int be = 0; be < 4; ++be) {
        ib[be] = __ldcg(&a.pidx[4 * pb + be]);
        wb[be] = __ldcg(&a.pw[4 * pb + be]);
      }
      for (int al = 0; al < 4; ++al) {
        const long row = (long)ca * a.n_sd + __ldcg(&a.pidx[4 * pa + al]);
        const double wa = __ldcg(&a.pw[4 * pa + al]);
        const double* brow = a.B0 + row * n2 + (long)cb * a.n_sd;
        double t = 0.0;
#pragma unroll
        for (int be = 0; be < 4; ++be) t += wb[be] * brow[ib[be]];
        acc += wa * t;
      }
      double kv = kscale * acc;
      const int ba = a.point_body[pa], bbd = a.point_body[pb];
      if (ba == bbd && a.bodies[ba].type == FSI_BODY_TORSIONAL)
        kv += (2.0 * a.ds / dt) / __ldcg(&a.st[ba].jac) * __ldcg(&a.sv[2 * pa + ca]) * __ldcg(&a.sv[2 * pb + cb]);
      a.K[(long)r * nf + cidx] = kv;
      a.K[(long)cidx * nf + r] = kv;
    }
    grid.sync();
    // ---- C: float factor in CTA 0, kSolves solves with double residuals computed by all CTAs
    float* Lf = reinterpret_cast<float*>(dyn_smem);  // [nf][ld]
    double* xs = reinterpret_cast<double*>(dyn_smem + (((size_t)nf * ld * 4 + 15) / 16) * 16);  // [nf]
    float* yv = reinterpret_cast<float*>(xs + nf);   // [nf]
    if (blockIdx.x == 0) {
      for (int i = tid >> 5; i < nf; i += nthr >> 5)
        for (int k = lane; k <= i; k += 32) Lf[(long)i * ld + k] = (float)__ldcg(&a.K[(long)i * nf + k]);
      __syncthreads();
      if (!chol_blocked(Lf, nf, ld, &sh_bad) && tid == 0) dev_set_status(a.status, FSI_ERR_NONFINITE);
      for (int i = tid; i < nf; i += nthr) xs[i] = 0.0;
    }
    for (int sidx = 0; sidx < kSolves; ++sidx) {
      if (blockIdx.x == 0) {
        const double* r = sidx == 0 ? a.rhs : res;
        for (int i = tid; i < nf; i += nthr) yv[i] = (float)__ldcg(&r[i]);
        __syncthreads();
        chol_solve(Lf, nf, ld, yv);
        for (int i = tid; i < nf; i += nthr) {
          xs[i] += (double)yv[i];
          a.f[i] = xs[i];
        }
        __syncthreads();
      }
      if (sidx == kSolves - 1) break;
      grid.sync();
      // residual r = rhs - K x in double, one warp per row
      {
        const long wg = gtid >> 5, nwg = gsize >> 5;
        for (long i = wg; i < nf; i += nwg) {
          double acc = 0.0;
          for (int k = lane; k < nf; k += 32) acc += __ldcg(&a.K[i * nf + k]) * __ldcg(&a.f[k]);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
          if (lane == 0) res[i] = __ldcg(&a.rhs[i]) - acc;
        }
      }
      grid.sync();
    }
    // ---- D: dtheta per torsional body (Eq. dtheta2), convergence on max |dtheta| (CTA 0)
    if (blockIdx.x == 0) {
      double dmax = 0.0;
      bool finite = true;
      for (int bi = 0; bi < a.n_bodies; ++bi) {
        const BodyDev b = a.bodies[bi];
        double part = 0.0;
        for (int p = b.off + tid; p < b.off + b.n; p += nthr) {
          part += __ldcg(&a.sv[2 * p]) * xs[p] + __ldcg(&a.sv[2 * p + 1]) * xs[nb + p];
          if (!isfinite(xs[p]) || !isfinite(xs[nb + p])) finite = false;
        }
        const double sf = block_sum(part, red);
        if (b.type == FSI_BODY_TORSIONAL && tid == 0) {
          BodyState& s = a.st[bi];
          const double dth = (s.r_phi - s.jac * s.theta_k + a.ds * sf) / s.jac;
          s.theta_k += dth;
          s.phi_k = 2.0 / dt * s.theta_k - s.r_theta;
          dmax = fmax(dmax, fabs(dth));
        }
      }
      if (!finite) dev_set_status(a.status, FSI_ERR_NONFINITE);
      if (tid == 0) {
        const int conv = (dmax <= a.tol) || !isfinite(dmax) || (*(volatile int*)a.status != 0);
        a.ctrl[0] = conv;
        a.ctrl[1] = it + 1;
      }
      __syncthreads();
    }
    grid.sync();
    if (tid == 0) sh_flag = *(volatile int*)&a.ctrl[0];
    __syncthreads();
    if (sh_flag) break;
    grid.sync();  // nobody may overwrite ctrl[0] before all CTAs have read it
  }

  // ---- Newmark update, forces, history (CTA 0)
  if (blockIdx.x == 0) {
    if (tid == 0 && !sh_flag) dev_set_status(a.status, FSI_ERR_NOT_CONVERGED);
    const int slot = a.ctrl[2] % a.hist_cap;
    for (int bi = 0; bi < a.n_bodies; ++bi) {
      const BodyDev b = a.bodies[bi];
      double px = 0.0, py = 0.0, pm = 0.0;
      for (int p = b.off + tid; p < b.off + b.n; p += nthr) {
        px += a.f[p];
        py += a.f[nb + p];
        pm += __ldcg(&a.sv[2 * p]) * a.f[p] + __ldcg(&a.sv[2 * p + 1]) * a.f[nb + p];
      }
      const double sx = block_sum(px, red), sy = block_sum(py, red), sm = block_sum(pm, red);
      if (tid == 0) {
        BodyState& s = a.st[bi];
        s.fx = a.ds * sx;
        s.fy = a.ds * sy;
        s.moment = b.type == FSI_BODY_TORSIONAL ? a.ds * sm : 0.0;
        if (b.type == FSI_BODY_TORSIONAL) {
          const double th_new = s.theta_k;
          const double ph_new = 2.0 / dt * th_new - s.r_theta;
          s.phidot = 4.0 / (dt * dt) * (th_new - s.theta) - 4.0 / dt * s.phi - s.phidot;
          s.theta = th_new;
          s.phi = ph_new;
        }
        double* hrow = a.hist + ((long)slot * a.n_bodies + bi) * 6;
        hrow[0] = s.fx;
        hrow[1] = s.fy;
        hrow[2] = s.moment;
        hrow[3] = b.type == FSI_BODY_TORSIONAL ? s.theta : 0.0;
        hrow[4] = b.type == FSI_BODY_TORSIONAL ? s.phi : 0.0;
        hrow[5] = (double)a.ctrl[1];
        if (!isfinite(s.fx) || !isfinite(s.fy)) dev_set_status(a.status, FSI_ERR_NONFINITE);
      }
    }
    if (tid == 0) a.ctrl[2] += 1;
  }
}

}  // namespace

size_t fsi_smem_bytes(int nf) {
  const size_t ld = (size_t)(nf | 1);
  return (((size_t)nf * ld * 4 + 15) / 16) * 16 + (size_t)nf * 12 + 64;
}

int fsi_kernel_max_ctas_per_sm(int nf) {
  cudaFuncSetAttribute(k_fsi, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fsi, 256, fsi_smem_bytes(nf));
  return n;
}

fsi_status launch_fsi(fsi_ctx* c) {
  FsiArgs a;
  a.s0 = c->s_all;
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
  a.max_iters = c->x.max_iters;
  a.n_sd = c->n_sd;
  a.ni = c->ni;
  a.nj = c->nj;
  a.i_lo = c->i_lo;
  a.j_lo = c->j_lo;
  a.B0 = c->B0;
  a.nb = c->nb;
  a.nf = c->nf;
  a.n_bodies = c->n_bodies;
  a.bodies = c->d_bodies;
  a.st = c->d_state;
  a.point_body = c->d_point_body;
  a.rpts = c->d_rpts;
  a.rur = c->d_rur;
  a.pidx = c->d_pidx;
  a.pw = c->d_pw;
  a.sv = c->d_sv;
  a.rhs = c->d_rhs;
  a.K = c->d_K;
  a.f = c->d_f;
  a.ctrl = c->d_ctrl;
  a.status = c->d_status;
  a.hist = c->d_hist;
  a.hist_cap = c->hist_cap;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->fsi_grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = fsi_smem_bytes(c->nf);
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  prof_mark(c, KC_FSI);
  FSI_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_fsi, a));
  prof_mark(c, KC_FSI);
  c->launches_per_step += 1;
  return FSI_OK;
}
