// FSI iteration of one time step (Algorithm 2; Eqs. stress2 and dtheta2) in double precision, as one
// cooperative kernel over a fixed set of CTAs:
//   A  body points at theta^(k), the hat map P (Eq. weights), rhs = P E0 (C s* + q_inf) - r^c(k)
//      + S^T (r^theta(k) - (2/dt) J^{-1} r^phidot(k))                                   [all CTAs]
//   B  K = (ds/h^2) P B0 P^T + (2 ds/dt) S^T J^{-1} S  (16 B0 lookups per entry)          [all CTAs]
//   C  f = K^{-1} rhs to double accuracy by iterative refinement: d = X r with a float inverse X,
//      f += d, r = rhs - K f in double, until |d| <= 1e-10 |f|                            [all CTAs]
//      X is carried across iterations and steps; each iteration first refreshes it for the new K with
//      two Newton-Schulz steps X <- 2X - X K X (tiled GEMMs over all CTAs; the error I - K X is squared
//      each time).  It is rebuilt from scratch (blocked float Cholesky and triangular inverse in CTA 0,
//      then W^T W over all CTAs) at the first step, when refinement stalls, or when it diverges.
//   D  dtheta = J^{-1}(r^phidot(k) + ds S f), convergence on max |dtheta| (every CTA computes the same
//      value in the same order, so all CTAs take the same branch without another barrier)
// repeated until max |dtheta| <= tol, then the Newmark update and force outputs (CTA 0).
// Data written by other CTAs inside this kernel is read with __ldcg (L2), so no stale L1 line is used.
#include <cooperative_groups.h>
#include <cmath>
#include "internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr int kMaxSolves = 8;         // refinement solves per attempt
constexpr double kStaleRatio = 0.02;  // |d_s| / |d_{s-1}| above this -> rebuild Kinv for the next iteration
constexpr double kRefineTol = 1e-10;  // stop at |d| <= 1e-10 |f|; the next correction would be ~ratio times that
constexpr int kNsSteps = 2;  // Newton-Schulz refreshes of the inverse per FSI iteration
constexpr int BS = 32;       // Cholesky / inverse / GEMM tile (one warp wide)
constexpr int kMaxBodies = 256;
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
  double* rhs;   // [nf] right-hand side, then [nf] residual
  double* K;     // [nf][nf] double, both triangles
  double* f;     // [nf]
  float* Xa;     // [nf][nf] float inverse of K, ping-pong buffer a
  float* Xb;     // [nf][nf] ping-pong buffer b (ctrl[7] says which one is current)
  float* S;      // [nf][nf] scratch: K X, or the inverse Cholesky factor during a rebuild
  double* part;  // [2 * gridDim] per-CTA maxima
  unsigned long long* phase_ns;  // [8] accumulated wall time per kernel phase
  int* ctrl;     // [1] iterations of the last step, [2] step index, [4] Kinv valid, [5] solves of the last
                 // step, [6] Kinv rebuilds so far, [8..11] vertex box touched by the corrector source
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

// Wall time per phase of the kernel, accumulated in nanoseconds (%globaltimer) by thread 0 of CTA 0 at the
// phase boundaries (after the grid barrier that ends the phase): 0 A, 1 B, 2 inverse refresh, 3 inverse
// rebuild, 4 refinement solves, 5 double residuals, 6 dtheta/convergence, 7 outputs.
struct PhaseClock {
  unsigned long long* acc;
  bool on;
  unsigned long long* last;
  __device__ PhaseClock(unsigned long long* a, bool o, unsigned long long* l) : acc(a), on(o && a), last(l) {
    if (on) *last = now();
  }
  __device__ static unsigned long long now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
  }
  __device__ void mark(int phase) {
    if (!on) return;
    const unsigned long long t = now();
    acc[phase] += t - *last;
    *last = t;
  }
};

// Deterministic block reductions (fixed tree); all threads must call; result valid in every thread.
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

__device__ double block_max(double x, double* red) {
  const int tid = threadIdx.x;
  red[tid] = x;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// C = A B (Xc == nullptr) or C = 2 Xc - A B for n x n row-major matrices, A given as double (Ad) or float
// (Af), B float.  32 x 32 output tiles are spread over the CTAs of the grid; each thread computes four
// entries of its tile.  sm: 32 * (n + 1) + 33 * n floats of shared memory.  All inputs may have been
// written earlier in the same launch, so they are read with __ldcg.
__device__ void gemm_tiles(int n, const double* __restrict__ Ad, const float* __restrict__ Af,
                           const float* __restrict__ B, const float* __restrict__ Xc, float* __restrict__ C,
                           float* sm) {
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  const int nt = (n + BS - 1) / BS;
  float* As = sm;
  const int lda = n + 1;
  float* Bs = sm + BS * lda;
  for (int t = blockIdx.x; t < nt * nt; t += gridDim.x) {
    const int ti = t / nt, tj = t - ti * nt;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    // whole 32 x n row panel of A and n x 32 column panel of B, loads issued back to back (unrolled) so
    // that many L2 round trips overlap
#pragma unroll 8
    for (int e = tid; e < BS * n; e += blockDim.x) {
      const int r = e / n, k = e - r * n;
      const int gi = ti * BS + r;
      float av = 0.0f;
      if (gi < n) av = Ad ? (float)__ldcg(&Ad[(long)gi * n + k]) : __ldcg(&Af[(long)gi * n + k]);
      As[r * lda + k] = av;
    }
#pragma unroll 8
    for (int e = tid; e < BS * n; e += blockDim.x) {
      const int k = e >> 5, c = e & 31;
      const int gj = tj * BS + c;
      Bs[k * (BS + 1) + c] = gj < n ? __ldcg(&B[(long)k * n + gj]) : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < n; ++k) {
      const float b = Bs[k * (BS + 1) + lane];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += As[(ty + 8 * q) * lda + k] * b;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gi = ti * BS + ty + 8 * q, gj = tj * BS + lane;
      if (gi < n && gj < n) C[(long)gi * n + gj] = Xc ? 2.0f * __ldcg(&Xc[(long)gi * n + gj]) - acc[q] : acc[q];
    }
  }
}

// Blocked right-looking Cholesky of the lower triangle of L (row stride ld) in shared memory.
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
    for (int i = jb + bs + tid; i < n; i += blockDim.x) {  // panel: X Ldiag^T = A
      float* row = L + (long)i * ld + jb;
      for (int c = 0; c < bs; ++c) {
        float v = row[c];
        const float* dr = L + (long)(jb + c) * ld + jb;
        for (int cc = 0; cc < c; ++cc) v -= row[cc] * dr[cc];
        row[c] = v / dr[c];
      }
    }
    __syncthreads();
    const int t0 = jb + bs;  // trailing update, one warp per row
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

// W = L^{-1} (lower triangular, float, row-major [n][n] in global memory) from the shared-memory factor.
// Diagonal blocks: one warp each, lane r holds row r (forward substitution with shuffles).  Off-diagonal
// blocks W_ij = -W_ii sum_{k=j}^{i-1} L_ik W_kj: one warp per block column j, rows i in order.
__device__ void tri_inverse(const float* L, int n, int ld, float* W) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int nblk = (n + BS - 1) / BS;
  for (long e = tid; e < (long)n * n; e += blockDim.x) W[e] = 0.0f;
  __syncthreads();
  for (int b = wid; b < nblk; b += nw) {
    const int jb = b * BS, bs = min(BS, n - jb);
    float a[BS], x[BS];
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      a[c] = (lane < bs && c <= lane && c < bs) ? L[(long)(jb + lane) * ld + jb + c] : 0.0f;
      x[c] = (c == lane) ? 1.0f : 0.0f;
    }
#pragma unroll
    for (int c = 0; c < BS; ++c)
      if (lane >= bs && c == lane) a[c] = 1.0f;
#pragma unroll
    for (int k = 0; k < BS; ++k) {
      if (lane == k) {
        const float inv = 1.0f / a[k];
#pragma unroll
        for (int c = 0; c < BS; ++c) x[c] *= inv;
      }
#pragma unroll
      for (int c = 0; c < BS; ++c) {
        const float xk = __shfl_sync(FULL, x[c], k);
        if (lane > k) x[c] -= a[k] * xk;
      }
    }
    if (lane < bs) {
#pragma unroll
      for (int c = 0; c < BS; ++c)
        if (c <= lane && c < bs) W[(long)(jb + lane) * n + jb + c] = x[c];
    }
  }
  __syncthreads();
  for (int bj = wid; bj < nblk; bj += nw) {
    const int jb = bj * BS, bsj = min(BS, n - jb);
    for (int bi = bj + 1; bi < nblk; ++bi) {
      const int ib = bi * BS, bsi = min(BS, n - ib);
      float t[BS];  // lane r: row ib + r of T = sum_k L_ik W_kj
#pragma unroll
      for (int c = 0; c < BS; ++c) t[c] = 0.0f;
      for (int bk = bj; bk < bi; ++bk) {
        const int kb = bk * BS, bsk = min(BS, n - kb);
        float wrow[BS];  // lane m: row kb + m of W_kj
#pragma unroll
        for (int c = 0; c < BS; ++c) wrow[c] = (lane < bsk && c < bsj) ? W[(long)(kb + lane) * n + jb + c] : 0.0f;
        for (int m = 0; m < bsk; ++m) {
          const float lim = lane < bsi ? L[(long)(ib + lane) * ld + kb + m] : 0.0f;
#pragma unroll
          for (int c = 0; c < BS; ++c) t[c] += lim * __shfl_sync(FULL, wrow[c], m);
        }
      }
      float wii[BS];  // lane r: row ib + r of W_ii
#pragma unroll
      for (int c = 0; c < BS; ++c) wii[c] = (lane < bsi && c < bsi) ? W[(long)(ib + lane) * n + ib + c] : 0.0f;
      float out[BS];
#pragma unroll
      for (int c = 0; c < BS; ++c) out[c] = 0.0f;
      for (int m = 0; m < bsi; ++m) {
#pragma unroll
        for (int c = 0; c < BS; ++c) out[c] -= wii[m] * __shfl_sync(FULL, t[c], m);
      }
      if (lane < bsi) {
#pragma unroll
        for (int c = 0; c < BS; ++c)
          if (c < bsj) W[(long)(ib + lane) * n + jb + c] = out[c];
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_fsi(FsiArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ double red[256];
  __shared__ double b_th[kMaxBodies], b_ph[kMaxBodies], b_rphi[kMaxBodies], b_rth[kMaxBodies], b_jac[kMaxBodies];
  __shared__ double b_tp[kMaxBodies];  // angle of the iterate that produced the current f (S, P of the solve)
  __shared__ int sh_bad;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const long gtid = (long)blockIdx.x * nthr + tid;
  const long gsize = (long)gridDim.x * nthr;
  const long wg = gtid >> 5, nwg = gsize >> 5;
  const int nb = a.nb, nf = a.nf;
  const int ld = nf | 1;
  const double dt = a.dt;
  double* res = a.rhs + nf;

  // per-CTA copy of the structural state (identical in every CTA)
  for (int bi = tid; bi < a.n_bodies; bi += nthr) {
    const BodyDev b = a.bodies[bi];
    const BodyState s = a.st[bi];
    if (b.type == FSI_BODY_TORSIONAL) {
      b_jac[bi] = 4.0 * b.inertia / (dt * dt) + 2.0 * b.damping / dt + b.stiffness;
      b_rphi[bi] = b.inertia * (4.0 * s.theta / (dt * dt) + 4.0 * s.phi / dt + s.phidot) +
                   b.damping * (2.0 * s.theta / dt + s.phi);
      b_rth[bi] = s.phi + 2.0 / dt * s.theta;
      b_th[bi] = s.theta;
      b_ph[bi] = s.phi;
      b_tp[bi] = s.theta;
    } else {
      b_jac[bi] = 1.0;
      b_rphi[bi] = b_rth[bi] = b_th[bi] = b_ph[bi] = b_tp[bi] = 0.0;
    }
  }
  int kinv_valid = *(volatile int*)&a.ctrl[4];
  int cur = *(volatile int*)&a.ctrl[7];
  float* gsm = reinterpret_cast<float*>(dyn_smem);  // GEMM tiles (all CTAs) / Cholesky factor (CTA 0)
  unsigned long long t_last = 0;
  PhaseClock clk(a.phase_ns, blockIdx.x == 0 && tid == 0, &t_last);
  __syncthreads();

  bool converged = false;
  int it = 0, solves_total = 0;
  for (; it < a.max_iters; ++it) {
    // ---- A: body points, P, right-hand side
    for (long p = gtid; p < nb; p += gsize) {
      const int bi = a.point_body[p];
      const BodyDev b = a.bodies[bi];
      double x, y, svx = 0.0, svy = 0.0, ucx, ucy, coef = 0.0;
      if (b.type == FSI_BODY_TORSIONAL) {
        const double th_k = b_th[bi], ph_k = b_ph[bi];
        const int j = (int)p - b.off;
        double sn, cs;
        sincos(b.theta0 + th_k, &sn, &cs);
        x = b.hx + (double)j * a.ds * cs;
        y = b.hy + (double)j * a.ds * sn;
        svx = (double)j * a.ds * (-sn);
        svy = (double)j * a.ds * cs;
        ucx = svx * ph_k;
        ucy = svy * ph_k;
        const double rphik = b_rphi[bi] - b_jac[bi] * th_k;
        const double rthk = b_rth[bi] - 2.0 / dt * th_k + ph_k;
        coef = rthk - 2.0 / dt * rphik / b_jac[bi];
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
      a.rhs[p] = ubx - ucx + svx * coef;
      a.rhs[nb + p] = uby - ucy + svy * coef;
    }
    grid.sync();
    clk.mark(0);
    // ---- B: K = (ds/h^2) P B0 P^T + (2 ds/dt) S^T J^{-1} S (both triangles written)
    {
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
        if (ba == bbd && a.bodies[ba].type == FSI_BODY_TORSIONAL) {
          const BodyDev b = a.bodies[ba];
          double sn, cs;
          sincos(b.theta0 + b_th[ba], &sn, &cs);
          const double sa = (double)(pa - b.off) * a.ds * (ca == 0 ? -sn : cs);
          const double sb = (double)(pb - b.off) * a.ds * (cb == 0 ? -sn : cs);
          kv += (2.0 * a.ds / dt) / b_jac[ba] * sa * sb;
        }
        a.K[(long)r * nf + cidx] = kv;
        a.K[(long)cidx * nf + r] = kv;
      }
    }
    grid.sync();
    clk.mark(1);
    // ---- C: refresh the float inverse (Newton-Schulz from the previous one, or a rebuild), then refine
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (kinv_valid) {
        for (int ns = 0; ns < kNsSteps; ++ns) {  // X <- 2X - X (K X): the error I - K X is squared
          const float* X = cur ? a.Xb : a.Xa;
          float* Xn = cur ? a.Xa : a.Xb;
          gemm_tiles(nf, a.K, nullptr, X, nullptr, a.S, gsm);  // S = K X
          grid.sync();
          gemm_tiles(nf, nullptr, X, a.S, X, Xn, gsm);         // Xn = 2 X - X S
          grid.sync();
          cur ^= 1;
        }
        clk.mark(2);
      } else {
        float* Lf = reinterpret_cast<float*>(dyn_smem);
        if (blockIdx.x == 0) {
          for (int i = tid >> 5; i < nf; i += nthr >> 5)
            for (int k = lane; k <= i; k += 32) Lf[(long)i * ld + k] = (float)__ldcg(&a.K[(long)i * nf + k]);
          __syncthreads();
          chol_blocked(Lf, nf, ld, &sh_bad);
          tri_inverse(Lf, nf, ld, a.S);
        }
        grid.sync();
        float* Xc = cur ? a.Xb : a.Xa;
        for (long i = wg; i < nf; i += nwg) {  // X = W^T W, warp per row i, lanes over k <= i
          for (int k0 = 0; k0 <= i; k0 += 32) {
            const int k = k0 + lane;
            float acc = 0.0f;
            if (k <= i)
              for (int m = (int)i; m < nf; ++m) acc += __ldcg(&a.S[(long)m * nf + i]) * __ldcg(&a.S[(long)m * nf + k]);
            if (k <= i) {
              Xc[i * nf + k] = acc;
              Xc[(long)k * nf + i] = acc;
            }
          }
        }
        grid.sync();
        kinv_valid = 1;
        if (blockIdx.x == 0 && tid == 0) a.ctrl[6] += 1;  // rebuild count
        clk.mark(3);
      }
      const float* Xinv = cur ? a.Xb : a.Xa;
      bool done = false, bad = false;
      int s = 0;
      double gd_prev = 0.0, worst_ratio = 0.0;
      for (; s < kMaxSolves; ++s) {
        double dmax = 0.0, xmax = 0.0;
        for (long i = wg; i < nf; i += nwg) {  // d = Kinv r, f += d
          const double* r = s == 0 ? a.rhs : res;
          float acc = 0.0f;
#pragma unroll 8
          for (int k = lane; k < nf; k += 32) acc += __ldcg(&Xinv[i * nf + k]) * (float)__ldcg(&r[k]);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
          if (lane == 0) {
            const double xi = (s == 0 ? 0.0 : a.f[i]) + (double)acc;
            a.f[i] = xi;
            dmax = fmax(dmax, fabs((double)acc));
            xmax = fmax(xmax, fabs(xi));
            if (!isfinite(xi)) dmax = INFINITY;
          }
        }
        dmax = block_max(dmax, red);
        xmax = block_max(xmax, red);
        if (tid == 0) {
          a.part[2 * blockIdx.x] = dmax;
          a.part[2 * blockIdx.x + 1] = xmax;
        }
        grid.sync();
        clk.mark(4);
        // every CTA reduces the per-CTA maxima the same way (one load per thread, fixed tree)
        const double gd = block_max(tid < (int)gridDim.x ? __ldcg(&a.part[2 * tid]) : 0.0, red);
        const double gx = block_max(tid < (int)gridDim.x ? __ldcg(&a.part[2 * tid + 1]) : 0.0, red);
        if (!isfinite(gd)) {  // a diverged inverse: rebuild and retry
          bad = true;
          break;
        }
        if (s > 0 && gd_prev > 0.0) worst_ratio = fmax(worst_ratio, gd / gd_prev);
        gd_prev = gd;
        if (gd <= kRefineTol * gx) {
          done = true;
          break;
        }
        if (s == kMaxSolves - 1) break;
        for (long i = wg; i < nf; i += nwg) {  // r = rhs - K f in double
          double acc = 0.0;
#pragma unroll 8
          for (int k = lane; k < nf; k += 32) acc += __ldcg(&a.K[i * nf + k]) * __ldcg(&a.f[k]);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
          if (lane == 0) res[i] = __ldcg(&a.rhs[i]) - acc;
        }
        grid.sync();
        clk.mark(5);
      }
      solves_total += s + 1;
      if (done) {
        if (worst_ratio > kStaleRatio) kinv_valid = 0;
        break;
      }
      kinv_valid = 0;  // not converged with this inverse: rebuild it and solve again
      if (attempt == 1 && blockIdx.x == 0 && tid == 0)
        dev_set_status(a.status, bad ? FSI_ERR_NONFINITE : FSI_ERR_NOT_CONVERGED);
    }
    // ---- D: dtheta per torsional body (Eq. dtheta2), convergence on max |dtheta| (same in every CTA)
    double dmax = 0.0;
    bool finite = true;
    for (int bi = 0; bi < a.n_bodies; ++bi) {
      const BodyDev b = a.bodies[bi];
      if (b.type != FSI_BODY_TORSIONAL) continue;
      double sn, cs;
      sincos(b.theta0 + b_th[bi], &sn, &cs);
      double part = 0.0;
      for (int p = b.off + tid; p < b.off + b.n; p += nthr) {
        const double q = (double)(p - b.off) * a.ds;
        const double fxp = __ldcg(&a.f[p]), fyp = __ldcg(&a.f[nb + p]);
        part += q * (-sn) * fxp + q * cs * fyp;
      }
      const double sf = block_sum(part, red);
      const double dth = (b_rphi[bi] - b_jac[bi] * b_th[bi] + a.ds * sf) / b_jac[bi];
      __syncthreads();
      if (tid == 0) {
        b_tp[bi] = b_th[bi];
        b_th[bi] += dth;
        b_ph[bi] = 2.0 / dt * b_th[bi] - b_rth[bi];
      }
      if (!isfinite(dth)) finite = false;
      dmax = fmax(dmax, fabs(dth));
      __syncthreads();
    }
    if (!finite && blockIdx.x == 0 && tid == 0) dev_set_status(a.status, FSI_ERR_NONFINITE);
    converged = (dmax <= a.tol) || !finite;
    clk.mark(6);
    if (converged) break;
    // No barrier here: after the last barrier of phase C only f is read (phase D), and the next write of
    // f comes after the phase-A and phase-B barriers of the next iteration.
  }

  // ---- Newmark update, forces, history (CTA 0)
  if (blockIdx.x == 0) {
    if (tid == 0 && !converged) dev_set_status(a.status, FSI_ERR_NOT_CONVERGED);
    const int slot = a.ctrl[2] % a.hist_cap;
    for (int bi = 0; bi < a.n_bodies; ++bi) {
      const BodyDev b = a.bodies[bi];
      double sn = 0.0, cs = 0.0;
      if (b.type == FSI_BODY_TORSIONAL) sincos(b.theta0 + b_tp[bi], &sn, &cs);  // S of the final solve
      double px = 0.0, py = 0.0, pm = 0.0;
      for (int p = b.off + tid; p < b.off + b.n; p += nthr) {
        const double fxp = __ldcg(&a.f[p]), fyp = __ldcg(&a.f[nb + p]);
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
          const double th_new = b_th[bi];
          const double ph_new = 2.0 / dt * th_new - b_rth[bi];
          s.phidot = 4.0 / (dt * dt) * (th_new - s.theta) - 4.0 / dt * s.phi - s.phidot;
          s.theta = th_new;
          s.phi = ph_new;
          s.theta_k = th_new;
          s.phi_k = ph_new;
        }
        double* hrow = a.hist + ((long)slot * a.n_bodies + bi) * 6;
        hrow[0] = s.fx;
        hrow[1] = s.fy;
        hrow[2] = s.moment;
        hrow[3] = b.type == FSI_BODY_TORSIONAL ? s.theta : 0.0;
        hrow[4] = b.type == FSI_BODY_TORSIONAL ? s.phi : 0.0;
        hrow[5] = (double)(it + 1);
        if (!isfinite(s.fx) || !isfinite(s.fy)) dev_set_status(a.status, FSI_ERR_NONFINITE);
      }
    }
    if (tid == 0) {
      a.ctrl[1] = it + 1;
      a.ctrl[2] += 1;
      a.ctrl[4] = kinv_valid;
      a.ctrl[7] = cur;
      a.ctrl[5] = solves_total;
    }
    // vertex box that the corrector source (E0^T P^T f, then curl) can touch: cells of the final P, grown
    // by the E0 support (1.5 cells), the hat support (1 cell) and the curl stencil (1 cell)
    int imin = 1 << 30, imax = -1, jmin = 1 << 30, jmax = -1;
    for (int p = tid; p < nb; p += nthr) {
      const int n0 = __ldcg(&a.pidx[4 * p]);
      const int ci = n0 % a.ni, cj = n0 / a.ni;
      imin = min(imin, ci);
      imax = max(imax, ci);
      jmin = min(jmin, cj);
      jmax = max(jmax, cj);
    }
    imin = -(int)block_max(-(double)imin, red);
    imax = (int)block_max((double)imax, red);
    jmin = -(int)block_max(-(double)jmin, red);
    jmax = (int)block_max((double)jmax, red);
    if (tid == 0) {
      a.ctrl[8] = a.i_lo + imin - 3;
      a.ctrl[9] = a.i_lo + imax + 4;
      a.ctrl[10] = a.j_lo + jmin - 3;
      a.ctrl[11] = a.j_lo + jmax + 4;
    }
    clk.mark(7);
  }
}

}  // namespace

size_t fsi_smem_bytes(int nf) {
  const size_t ld = (size_t)(nf | 1);
  const size_t chol = (((size_t)nf * ld * 4 + 15) / 16) * 16;
  const size_t gemm = ((size_t)BS * (nf + 1) + (size_t)(BS + 1) * nf) * 4;
  return (chol > gemm ? chol : gemm) + 64;
}

int fsi_kernel_max_ctas_per_sm(int nf) {
  cudaFuncSetAttribute(k_fsi, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
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
  a.rhs = c->d_rhs;
  a.K = c->d_K;
  a.f = c->d_f;
  a.Xa = c->d_Kinv;
  a.Xb = c->d_W;
  a.S = c->d_S;
  a.part = c->d_part;
  a.ctrl = c->d_ctrl;
  a.phase_ns = c->d_phase;
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
