// Deformable body (Sec. 2.1 Eq. beam; App. A with J_d, S_d): device routines of the FSI kernel.
//
// The flag is a chain of two-dimensional corotational Euler-Bernoulli beam elements (Crisfield, Non-linear
// Finite Element Analysis of Solids and Structures, vol. 1, ch. 7) whose nodes are the body points; node 0
// is clamped.  Element a-b with chord length L, unit chord (c, s), chord rotation psi from the undeformed
// direction, local rotations tb = theta - psi, stretch u = L - L0:
//   N = (EA/L0) u,  Ma = (2EI/L0)(2 tb_a + tb_b),  Mb = (2EI/L0)(tb_a + 2 tb_b)
//   f_a = (-(N c + Q s), Q c - N s, Ma),  f_b = (N c + Q s, N s - Q c, Mb),  Q = (Ma + Mb)/L
//   K = ka r r^T + kb (2 ga ga^T + ga gb^T + gb ga^T + 2 gb gb^T) + (N/L) z z^T + (Q/L)(r z^T + z r^T)
// with ka = EA/L0, kb = 2EI/L0, r = (-c,-s,0,c,s,0), z = (s,-c,0,-s,c,0), ga = e_a - z/L, gb = e_b - z/L.
//
// Precision (GB300 runs FP64 at 1/64 of the FP32 rate and ~64 cycles per dependent FP64 instruction):
// the internal forces and the structural residual r^zeta(k) are FP64, because the fixed point of the FSI
// iteration is defined by them; J_d = 4M/dt^2 + K is assembled, factored and solved in FP32.  A different
// J_d changes only the path of the iteration: at its fixed point J_d^-1 (r^zeta + ds T^T f) = 0, and the
// terms that J_d^-1 adds to the small matrix and to its right-hand side cancel.  The kernel applies the
// FP32 solves only to residuals that vanish at the fixed point (r^zeta + ds T^T f_prev), so their float
// errors vanish there too.  With the Jacobi-scaled condition number of J_d of a few tens, the FP32 solves
// are accurate to ~1e-7 relative.
//
// J_d is block tridiagonal (3 x 3 blocks: D_i on the diagonal, B_i = J_{i+1,i} below it) and is factored
// from both ends at once (two lanes of one warp in lockstep, m = (N-1)/2 the meeting block):
//   top     S_0 = D_0,      F_i = B_i S_i^-1,        S_{i+1} = D_{i+1} - F_i B_i^T          (i < m)
//   bottom  T_{N-1} = D_{N-1}, H_{i-1} = B_{i-1}^T T_i^-1, T_{i-1} = D_{i-1} - H_{i-1} B_{i-1} (i > m)
//   middle  Z = S_m + T_m - D_m
// and a solve J x = b runs forward from both ends (y_i = b_i - F_{i-1} y_{i-1}, w_i = b_i - H_i w_{i+1}),
// takes x_m = Z^-1 (y_m + w_m - b_m), then substitutes back outwards (x_i = S_i^-1 (y_i - B_i^T x_{i+1}),
// x_i = T_i^-1 (w_i - B_{i-1} x_{i-1})): chains of about N/2 block steps instead of N.
#pragma once
#include <cmath>
#include "internal.h"

namespace beam {

// 1/sqrt(x) in double: single-precision seed, then two Newton steps r <- r (3 - x r^2) / 2
__device__ __forceinline__ double rsqrt_d(double x) {
  const double hx = -0.5 * x;
  double r = (double)rsqrtf((float)x);
  r = r * fma(hx * r, r, 1.5);
  r = r * fma(hx * r, r, 1.5);
  return r;
}

// Angle from the unit reference chord (cr, sr) to the unit chord (c, s).  Within a time step the chord
// turns by far less than 0.02 rad, where the arcsine series x + x^3/6 + 3x^5/40 + 5x^7/112 of the cross
// product is exact to double rounding; otherwise atan2.
__device__ __forceinline__ double chord_rotation(double cr, double sr, double c, double s) {
  const double x = cr * s - sr * c;
  const double co = cr * c + sr * s;
  if (fabs(x) < 0.02 && co > 0.0) {
    const double x2 = x * x;
    double p = fma(x2, 5.0 / 112.0, 3.0 / 40.0);
    p = fma(p, x2, 1.0 / 6.0);
    return fma(x * x2, p, x);
  }
  return atan2(x, co);
}

// Symmetric 3 x 3 blocks are stored as [00, 01, 02, 11, 12, 22]; full blocks row-major.
__host__ __device__ __forceinline__ int sidx(int p, int q) {
  const int a = p < q ? p : q, b = p < q ? q : p;
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

// One element: FP64 end forces from the end nodes (x, y, theta) and the reference chord of the step
// (psi_r, cr, sr); FP32 tangent blocks aa (sym), bb (sym), ba (full, rows b-dofs, columns a-dofs).
struct ElemParams {
  double L0, ka, kb;  // undeformed length, EA/L0, 2EI/L0
};
__device__ __forceinline__ void element(const ElemParams& P, double xa, double ya, double ta, double xb, double yb,
                                        double tb, double psi_r, double cr, double sr, double fa[3], double fb[3],
                                        float kaa[6], float kbb[6], float kba[9]) {
  const double dx = xb - xa, dy = yb - ya;
  const double L2 = fma(dx, dx, dy * dy);
  const double il = rsqrt_d(L2);
  const double c = dx * il, s = dy * il;
  const double L = L2 * il;
  const double psi = psi_r + chord_rotation(cr, sr, c, s);
  const double tba = ta - psi, tbb = tb - psi;
  const double N = P.ka * (L - P.L0);
  const double Ma = P.kb * fma(2.0, tba, tbb), Mb = P.kb * fma(2.0, tbb, tba);
  const double Q = (Ma + Mb) * il;
  const double fx = fma(N, c, Q * s), fy = fma(Q, c, -N * s);
  fa[0] = -fx;
  fa[1] = fy;
  fa[2] = Ma;
  fb[0] = fx;
  fb[1] = -fy;
  fb[2] = Mb;
  // tangent in FP32
  const float cf = (float)c, sf = (float)s, ilf = (float)il;
  const float ka = (float)P.ka, kb = (float)P.kb, nl = (float)(N * il), ql = (float)(Q * il);
  const float r[6] = {-cf, -sf, 0.f, cf, sf, 0.f};
  const float z[6] = {sf, -cf, 0.f, -sf, cf, 0.f};
  const float ga[6] = {-sf * ilf, cf * ilf, 1.f, sf * ilf, -cf * ilf, 0.f};
  const float gb[6] = {-sf * ilf, cf * ilf, 0.f, sf * ilf, -cf * ilf, 1.f};
  auto Kpq = [&](int p, int q) {
    return ka * r[p] * r[q] + kb * (2.f * ga[p] * ga[q] + ga[p] * gb[q] + gb[p] * ga[q] + 2.f * gb[p] * gb[q]) +
           nl * z[p] * z[q] + ql * (r[p] * z[q] + z[p] * r[q]);
  };
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = p; q < 3; ++q) {
      kaa[sidx(p, q)] = Kpq(p, q);
      kbb[sidx(p, q)] = Kpq(p + 3, q + 3);
    }
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) kba[3 * p + q] = Kpq(p + 3, q);
}

// --- 3 x 3 float block helpers -------------------------------------------------------------------------

__device__ __forceinline__ void inv3s(const float S[6], float Si[6]) {
  const float c00 = S[3] * S[5] - S[4] * S[4];
  const float c01 = S[2] * S[4] - S[1] * S[5];
  const float c02 = S[1] * S[4] - S[2] * S[3];
  const float c11 = S[0] * S[5] - S[2] * S[2];
  const float c12 = S[1] * S[2] - S[0] * S[4];
  const float c22 = S[0] * S[3] - S[1] * S[1];
  const float id = 1.0f / (S[0] * c00 + S[1] * c01 + S[2] * c02);
  Si[0] = c00 * id;
  Si[1] = c01 * id;
  Si[2] = c02 * id;
  Si[3] = c11 * id;
  Si[4] = c12 * id;
  Si[5] = c22 * id;
}

// E = Bk * Si (full x sym)
__device__ __forceinline__ void mul_fs(const float Bk[9], const float Si[6], float E[9]) {
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      E[3 * p + q] = Bk[3 * p] * Si[sidx(0, q)] + Bk[3 * p + 1] * Si[sidx(1, q)] + Bk[3 * p + 2] * Si[sidx(2, q)];
}

// S = D - E * Bk^T (symmetric result)
__device__ __forceinline__ void schur(const float D[6], const float E[9], const float Bk[9], float S[6]) {
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = p; q < 3; ++q)
      S[sidx(p, q)] =
          D[sidx(p, q)] - (E[3 * p] * Bk[3 * q] + E[3 * p + 1] * Bk[3 * q + 1] + E[3 * p + 2] * Bk[3 * q + 2]);
}

__device__ __forceinline__ void load_block(const float* src, bool transpose, float out[9]) {
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) out[3 * p + q] = transpose ? src[3 * q + p] : src[3 * p + q];
}

// Factor arrays of one body (shared memory, N blocks): Mi[N][6] (D_i on entry; S_i^-1 / T_i^-1 on exit,
// entry m then holds Z^-1 through Zi), Bm[N][9] (B_i, i < N-1), Em[N][9] (F_i for i < m, H_i for
// m <= i < N-1).
struct Factor {
  float* Mi;
  const float* Bm;
  float* Em;
  float* Zi;
  int N;
};

__host__ __device__ __forceinline__ int meet(int N) { return (N - 1) / 2; }

// Twisted factorization: lanes 0 (top) and 1 (bottom) of the calling warp; the other lanes only join the
// shuffle.  The whole warp must call.
__device__ inline void factor(const Factor& F) {
  const int lane = threadIdx.x & 31;
  const int N = F.N, m = meet(N);
  const bool top = lane == 0;
  const int steps = top ? m : N - 1 - m;
  const int nmax = N - 1 - m;  // >= m
  float S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, Dm[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int i0 = top ? 0 : N - 1;
  if (lane < 2) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      S[k] = F.Mi[6 * i0 + k];
      Dm[k] = F.Mi[6 * m + k];
    }
  }
  for (int t = 0; t < nmax; ++t) {
    if (lane < 2 && t < steps) {
      const int i = top ? t : N - 1 - t;
      const int nx = top ? i + 1 : i - 1;
      float Si[6], Bk[9], E[9], Dn[6];
      load_block(F.Bm + 9 * (top ? i : i - 1), !top, Bk);
#pragma unroll
      for (int k = 0; k < 6; ++k) Dn[k] = F.Mi[6 * nx + k];
      inv3s(S, Si);
      mul_fs(Bk, Si, E);
      schur(Dn, E, Bk, S);
#pragma unroll
      for (int k = 0; k < 6; ++k) F.Mi[6 * i + k] = Si[k];
#pragma unroll
      for (int k = 0; k < 9; ++k) F.Em[9 * (top ? i : i - 1) + k] = E[k];
    }
  }
  // Z = S_m + T_m - D_m (lane 1 hands T_m to lane 0)
  float Z[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float tm = __shfl_down_sync(0xffffffffu, S[k], 1);
    Z[k] = S[k] + tm - Dm[k];
  }
  if (lane == 0) {
    float Zi[6];
    inv3s(Z, Zi);
#pragma unroll
    for (int k = 0; k < 6; ++k) F.Zi[k] = Zi[k];
  }
  __syncwarp();
}

// Solve J x = b for RHS r = lane / 2 < nrhs (lanes 2r: top, 2r+1: bottom) in place: Y[r] (stride ldy,
// 3N floats) holds b on entry and x on exit.  The whole warp must call; Mi, Bm, Em, Zi from factor().
__device__ inline void solve(const Factor& F, float* Y, int ldy, int nrhs) {
  const int lane = threadIdx.x & 31;
  const int N = F.N, m = meet(N);
  const int rr = lane >> 1;
  const bool top = (lane & 1) == 0;
  const bool act = rr < nrhs;
  float* y = Y + (long)(act ? rr : 0) * ldy;
  const int steps = top ? m : N - 1 - m;
  const int nmax = N - 1 - m;
  float v[3] = {0.f, 0.f, 0.f}, bm[3] = {0.f, 0.f, 0.f};
  const int i0 = top ? 0 : N - 1;
  if (act) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      v[k] = y[3 * i0 + k];
      bm[k] = y[3 * m + k];
    }
  }
  for (int t = 0; t < nmax; ++t) {  // forward from both ends
    if (act && t < steps) {
      const int i = top ? t + 1 : N - 2 - t;  // block being reduced
      const float* E = F.Em + 9 * (top ? i - 1 : i);
      float b[3], nv[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) b[k] = y[3 * i + k];
#pragma unroll
      for (int p = 0; p < 3; ++p) nv[p] = b[p] - (E[3 * p] * v[0] + E[3 * p + 1] * v[1] + E[3 * p + 2] * v[2]);
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = nv[k];
      if (i != m) {
#pragma unroll
        for (int k = 0; k < 3; ++k) y[3 * i + k] = v[k];
      }
    }
  }
  // middle block: x_m = Z^-1 (y_m + w_m - b_m); the bottom lane's w_m comes by shuffle
  float xm[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float w = __shfl_down_sync(0xffffffffu, v[k], 1);
    xm[k] = v[k] + w - bm[k];
  }
  float x[3];
#pragma unroll
  for (int p = 0; p < 3; ++p) x[p] = F.Zi[sidx(p, 0)] * xm[0] + F.Zi[sidx(p, 1)] * xm[1] + F.Zi[sidx(p, 2)] * xm[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) x[k] = __shfl_sync(0xffffffffu, x[k], lane & ~1);
  if (act && top) {
#pragma unroll
    for (int k = 0; k < 3; ++k) y[3 * m + k] = x[k];
  }
  for (int t = 0; t < nmax; ++t) {  // back substitution outwards
    if (act && t < steps) {
      const int i = top ? m - 1 - t : m + 1 + t;
      float C[9];
      load_block(F.Bm + 9 * (top ? i : i - 1), top, C);  // top: B_i^T, bottom: B_{i-1}
      const float* Si = F.Mi + 6 * i;
      float g[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) g[p] = y[3 * i + p] - (C[3 * p] * x[0] + C[3 * p + 1] * x[1] + C[3 * p + 2] * x[2]);
#pragma unroll
      for (int p = 0; p < 3; ++p) x[p] = Si[sidx(p, 0)] * g[0] + Si[sidx(p, 1)] * g[1] + Si[sidx(p, 2)] * g[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) y[3 * i + k] = x[k];
    }
  }
  __syncwarp();
}

// --- one flag's linearisation at chi^(k), run by threads t = 0..nt-1 of a group that synchronises between
// the two passes (the caller passes its barrier) --------------------------------------------------------

struct Flag {
  int N;                                  // elements (free nodes)
  double hx, hy;                          // clamp
  double mu, ds;                          // mass per length, element length
  ElemParams P;                           // L0, EA/L0, 2EI/L0
  double four_dt2, four_dt;               // 4/dt^2, 4/dt
  const double* chi;                      // [3N] iterate chi^(k)
  const double* ref;                      // [N][3] reference chord of the step: psi, c, s
  const double *chi_n, *zeta_n, *zdot_n;  // [3N] state of step n
  double* fab;                            // [N][6] element end forces (scratch)
  float* ey;                              // [N][12] element tangents (scratch; [Em | y] after the factorization)
  float* mi;                              // [N][6] D_i (assembly), factor blocks afterwards
  float* bm;                              // [N][9] B_i
  double* rz;                             // [3N] r^zeta(k)
  float* y0;                              // [3N] first right-hand side r^zeta(k) + ds T^T f (float), or NULL
  const double* f;                        // surface stress of nodes 1..N: x at f[i], y at f[fstride + i]; or NULL
  int fstride;
};

// Pass 1: element end forces (FP64) and tangent blocks (FP32).
__device__ inline void flag_elements(const Flag& F, int t, int nt) {
  for (int e = t; e < F.N; e += nt) {
    double xa = F.hx, ya = F.hy, ta = 0.0;
    if (e > 0) {
      xa = F.chi[3 * (e - 1)];
      ya = F.chi[3 * (e - 1) + 1];
      ta = F.chi[3 * (e - 1) + 2];
    }
    const double* rf = F.ref + 3 * e;
    double fa[3], fb[3];
    float kaa[6], kbb[6], kba[9];
    element(F.P, xa, ya, ta, F.chi[3 * e], F.chi[3 * e + 1], F.chi[3 * e + 2], rf[0], rf[1], rf[2], fa, fb, kaa, kbb,
            kba);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      F.fab[6 * e + k] = fa[k];
      F.fab[6 * e + 3 + k] = fb[k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      F.ey[12 * e + k] = kaa[k];
      F.ey[12 * e + 6 + k] = kbb[k];
    }
    if (e > 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) F.bm[9 * (e - 1) + k] = kba[k];
    }
  }
}

// Pass 2 (after a barrier): diagonal blocks D_i = K_bb(element i) + K_aa(element i+1) + 4M_i/dt^2 and
// r^zeta(k) = M ((4/dt^2)(chi_n - chi^(k)) + (4/dt) zeta_n + zetadot_n) - R(chi^(k)) per free node i.
__device__ inline void flag_assemble(const Flag& F, int t, int nt) {
  const int N = F.N;
  for (int i = t; i < N; i += nt) {
    const double mt = F.mu * F.ds * (i == N - 1 ? 0.5 : 1.0);
    const double mr = mt * F.ds * F.ds * (1.0 / 12.0);
    float D[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) D[k] = F.ey[12 * i + 6 + k] + (i + 1 < N ? F.ey[12 * (i + 1) + k] : 0.f);
    D[0] += (float)(F.four_dt2 * mt);
    D[3] += (float)(F.four_dt2 * mt);
    D[5] += (float)(F.four_dt2 * mr);
#pragma unroll
    for (int k = 0; k < 6; ++k) F.mi[6 * i + k] = D[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int g = 3 * i + k;
      double R = F.fab[6 * i + 3 + k];
      if (i + 1 < N) R += F.fab[6 * (i + 1) + k];
      const double rz =
          (k < 2 ? mt : mr) * (F.four_dt2 * (F.chi_n[g] - F.chi[g]) + F.four_dt * F.zeta_n[g] + F.zdot_n[g]) - R;
      F.rz[g] = rz;
      if (F.y0) F.y0[g] = (float)(k < 2 && F.f ? rz + F.ds * F.f[k * F.fstride + i] : rz);
    }
  }
}

__device__ __forceinline__ Factor flag_factor_view(const Flag& F) {
  return Factor{F.mi, F.bm, F.ey, F.mi + 6 * meet(F.N), F.N};
}

}  // namespace beam
