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
// J_d is block tridiagonal (3 x 3 blocks: D_i on the diagonal, R_i = J_{i,i+1} to the right) and is factored
// by block cyclic reduction (a block Cholesky factorization in nested-dissection order): at level l
// (stride s = 2^l) the active rows are those with (i + 1) % s == 0; every other one ((i + 1)/s odd) is
// eliminated, in parallel, and its two active neighbours k absorb it:
//   D_k -= J_{k,r} D_r^-1 J_{r,k},   R_k <- -J_{k,r'} D_{r'}^-1 J_{r',k+2s}     (r = k - s, r' = k + s)
// until the one row left at the top has no neighbour.  A solve reduces the right-hand sides level by level
// (b_k -= J_{k,r} D_r^-1 b_r) and substitutes back from the top (x_r = D_r^-1 (b_r - J_{r,r-s} x_{r-s}
// - J_{r,r+s} x_{r+s})).  The dependent chain is about 2 log2(N) parallel steps, where a sequential
// (Thomas or twisted) factorization has N or N/2: measured on GB300 a sequential 3 x 3 block step costs
// ~200 cycles of latency, so the chain length is what sets the time.
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
  const float id = __frcp_rn(S[0] * c00 + S[1] * c01 + S[2] * c02);
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

// Block cyclic reduction arrays of one flag (shared memory, N blocks):
//   D[N][6]  diagonal blocks (symmetric); replaced by their inverse at the level the row is eliminated
//   R[N][9]  R_i = J_{i,i+s} for the current level (zero where there is no right neighbour); frozen once
//            row i is eliminated
//   L[N][9]  L_i = J_{i,i-s} at the level row i is eliminated (copied before the left neighbour moves on)
struct Bcr {
  float* D;
  float* R;
  float* L;
  int N;
};

__device__ __forceinline__ void load9(const float* p, float a[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) a[k] = p[k];
}
__device__ __forceinline__ void load6(const float* p, float a[6]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) a[k] = p[k];
}

// Rows of level s (a power of two): eliminated i = (2m + 1) s - 1, kept k = (2m + 2) s - 1 (m = 0, 1, ...).

// Factorization, by threads t = 0..nt-1 of a group with barrier sync() (all of them must call).
template <class Sync>
__device__ __forceinline__ void bcr_factor(const Bcr& B, int t, int nt, Sync sync) {
  const int N = B.N;
  for (int s = 1; s <= N; s <<= 1) {
    const int n_el = (N / s + 1) >> 1;  // rows (2m+1)s - 1 < N
    for (int mm = t; mm < n_el; mm += nt) {  // eliminated rows: invert D, keep J_{i,i-s}
      const int i = (2 * mm + 1) * s - 1;
      float d[6], di[6];
      load6(B.D + 6 * i, d);
      inv3s(d, di);
#pragma unroll
      for (int k = 0; k < 6; ++k) B.D[6 * i + k] = di[k];
      if (i - s >= 0) {
        float r[9];
        load9(B.R + 9 * (i - s), r);  // J_{i-s,i}
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int q = 0; q < 3; ++q) B.L[9 * i + 3 * p + q] = r[3 * q + p];
      } else {  // no left neighbour: zero, so that the solve may read it with weight zero
#pragma unroll
        for (int k = 0; k < 9; ++k) B.L[9 * i + k] = 0.f;
      }
    }
    sync();
    const int n_kept = N / (2 * s);  // rows (2m+2)s - 1 < N
    for (int mm = t; mm < n_kept; mm += nt) {  // kept rows absorb their eliminated neighbours
      const int k = (2 * mm + 2) * s - 1;
      const int r = k - s, r2 = k + s;
      float d[6], rr[9], dinv[6];
      load6(B.D + 6 * k, d);
      load9(B.R + 9 * r, rr);  // J_{r,k}
      load6(B.D + 6 * r, dinv);
      {  // D_k -= J_{k,r} Dinv_r J_{r,k} = rr^T Dinv rr
        float a[9];  // a = Dinv rr
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int q = 0; q < 3; ++q)
            a[3 * p + q] = dinv[sidx(p, 0)] * rr[q] + dinv[sidx(p, 1)] * rr[3 + q] + dinv[sidx(p, 2)] * rr[6 + q];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int q = p; q < 3; ++q) d[sidx(p, q)] -= rr[p] * a[q] + rr[3 + p] * a[3 + q] + rr[6 + p] * a[6 + q];
      }
      float nr[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (r2 < N) {
        float rk[9], dinv2[6], e[9];
        load9(B.R + 9 * k, rk);  // J_{k,r2}
        load6(B.D + 6 * r2, dinv2);
        mul_fs(rk, dinv2, e);  // e = J_{k,r2} Dinv_{r2}
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int q = p; q < 3; ++q)
            d[sidx(p, q)] -= e[3 * p] * rk[3 * q] + e[3 * p + 1] * rk[3 * q + 1] + e[3 * p + 2] * rk[3 * q + 2];
        if (k + 2 * s < N) {  // new coupling J_{k,k+2s} = -e J_{r2,r2+s}
          float r2r[9];
          load9(B.R + 9 * r2, r2r);
#pragma unroll
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q)
              nr[3 * p + q] = -(e[3 * p] * r2r[q] + e[3 * p + 1] * r2r[3 + q] + e[3 * p + 2] * r2r[6 + q]);
        }
      }
#pragma unroll
      for (int k2 = 0; k2 < 6; ++k2) B.D[6 * k + k2] = d[k2];
#pragma unroll
      for (int k2 = 0; k2 < 9; ++k2) B.R[9 * k + k2] = nr[k2];
    }
    sync();
  }
}

// y_out = S y for symmetric S
__device__ __forceinline__ void symv(const float S[6], const float y[3], float out[3]) {
#pragma unroll
  for (int p = 0; p < 3; ++p) out[p] = S[sidx(p, 0)] * y[0] + S[sidx(p, 1)] * y[1] + S[sidx(p, 2)] * y[2];
}

// Solve J x = b for nrhs <= 8 right-hand sides Y[j] (stride ldy, 3N floats each; b on entry, x on exit) with
// the factor of bcr_factor, by threads t = 0..nt-1 of a group with barrier sync() (all of them must call;
// nt a multiple of 8).  Each (row, right-hand side) pair of a level is one thread's work item; a missing
// neighbour is read at a valid index with weight zero so that both neighbours' loads issue at once.
template <class Sync>
__device__ __forceinline__ void bcr_solve(const Bcr& B, float* Y, int ldy, int nrhs, int t, int nt, Sync sync) {
  const int N = B.N;
  int top = 1;
  while (top * 2 <= N) top <<= 1;
  // work mapping: one right-hand side -> all threads on rows; several -> 8 groups, group j = right-hand side j
  const int j = nrhs == 1 ? 0 : (t & 7);
  const int m0 = nrhs == 1 ? t : (t >> 3), dm = nrhs == 1 ? nt : (nt >> 3);
  const bool on = j < nrhs;
  float* y = Y + (long)(on ? j : 0) * ldy;
  for (int s = 1; s <= N; s <<= 1) {  // reduction: kept rows take b_k -= J_{k,r} Dinv_r b_r from both sides
    const int n_kept = N / (2 * s);
    for (int mm = m0; on && mm < n_kept; mm += dm) {
      const int k = (2 * mm + 2) * s - 1;
      const int r = k - s, r2 = k + s;
      const bool has2 = r2 < N;
      const int q2 = has2 ? r2 : r;
      float d1[6], c1[9], y1[3], d2[6], c2[9], y2[3], bk[3];
      load6(B.D + 6 * r, d1);
      load9(B.R + 9 * r, c1);  // J_{r,k}; J_{k,r} = c1^T
      load6(B.D + 6 * q2, d2);
      load9(B.L + 9 * q2, c2);  // J_{r2,k}; J_{k,r2} = c2^T
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        y1[p] = y[3 * r + p];
        y2[p] = y[3 * q2 + p];
        bk[p] = y[3 * k + p];
      }
      const float w2 = has2 ? 1.f : 0.f;
      float u1[3], u2[3];
      symv(d1, y1, u1);
      symv(d2, y2, u2);
#pragma unroll
      for (int p = 0; p < 3; ++p)
        y[3 * k + p] = bk[p] - (c1[p] * u1[0] + c1[3 + p] * u1[1] + c1[6 + p] * u1[2]) -
                       w2 * (c2[p] * u2[0] + c2[3 + p] * u2[1] + c2[6 + p] * u2[2]);
    }
    sync();
  }
  for (int s = top; s >= 1; s >>= 1) {  // back substitution from the top level down
    const int n_el = (N / s + 1) >> 1;
    for (int mm = m0; on && mm < n_el; mm += dm) {
      const int r = (2 * mm + 1) * s - 1;
      const bool has1 = r - s >= 0, has2 = r + s < N;
      const int k1 = has1 ? r - s : r, k2 = has2 ? r + s : r;
      float cl[9], cr[9], di[6], g[3], x1[3], x2[3];
      load9(B.L + 9 * r, cl);
      load9(B.R + 9 * r, cr);
      load6(B.D + 6 * r, di);
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        g[p] = y[3 * r + p];
        x1[p] = y[3 * k1 + p];
        x2[p] = y[3 * k2 + p];
      }
      const float w1 = has1 ? 1.f : 0.f, w2 = has2 ? 1.f : 0.f;
#pragma unroll
      for (int p = 0; p < 3; ++p)
        g[p] -= w1 * (cl[3 * p] * x1[0] + cl[3 * p + 1] * x1[1] + cl[3 * p + 2] * x1[2]) +
                w2 * (cr[3 * p] * x2[0] + cr[3 * p + 1] * x2[1] + cr[3 * p + 2] * x2[2]);
      float x[3];
      symv(di, g, x);
#pragma unroll
      for (int p = 0; p < 3; ++p) y[3 * r + p] = x[p];
    }
    sync();
  }
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
  const double* cn;                       // [3N] M ((4/dt^2) chi_n + (4/dt) zeta_n + zetadot_n), r^zeta_n
  double* fab;                            // [N][6] element end forces (scratch)
  float* ey;                              // [N][12] element tangents (scratch; [L | y] after the factorization)
  float* mi;                              // [N][6] D_i (assembly), factor blocks afterwards
  float* bm;                              // [N][9] R_i = J_{i,i+1}
  double* rz;                             // [3N] r^zeta(k)
  float* y0;                              // [3N] first right-hand side r^zeta(k) + ds T^T f (float), or NULL
  const double* f;                        // surface stress of nodes 1..N: x at f[i], y at f[fstride + i]; or NULL
  int fstride;
};

// Pass 1: element end forces (FP64) and tangent blocks (FP32).
__device__ __forceinline__ void flag_elements(const Flag& F, int t, int nt) {
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
    if (e > 0) {  // R_{e-1} = J_{e-1,e} (free nodes) = K_ab = K_ba^T of element e
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) F.bm[9 * (e - 1) + 3 * p + q] = kba[3 * q + p];
    }
  }
}

// Lumped mass of free node i (of N) for dof k: mass_per_length * ds (half at the tip) on the translations,
// times ds^2/12 on the rotation.
__host__ __device__ __forceinline__ double node_mass(double mu, double ds, int N, int i, int k) {
  const double mt = mu * ds * (i == N - 1 ? 0.5 : 1.0);
  return k < 2 ? mt : mt * ds * ds * (1.0 / 12.0);
}

// Pass 2 (after a barrier): diagonal blocks D_i = K_bb(element i) + K_aa(element i+1) + 4M_i/dt^2 and
// r^zeta(k) = r^zeta_n - (4/dt^2) M chi^(k) - R(chi^(k)) per free node i (App. A).
__device__ __forceinline__ void flag_assemble(const Flag& F, int t, int nt) {
  const int N = F.N;
  for (int i = t; i < N; i += nt) {
    const double mt = node_mass(F.mu, F.ds, N, i, 0), mr = node_mass(F.mu, F.ds, N, i, 2);
    float D[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) D[k] = F.ey[12 * i + 6 + k] + (i + 1 < N ? F.ey[12 * (i + 1) + k] : 0.f);
    D[0] += (float)(F.four_dt2 * mt);
    D[3] += (float)(F.four_dt2 * mt);
    D[5] += (float)(F.four_dt2 * mr);
#pragma unroll
    for (int k = 0; k < 6; ++k) F.mi[6 * i + k] = D[k];
    if (i == N - 1) {  // the tip has no right neighbour
#pragma unroll
      for (int k = 0; k < 9; ++k) F.bm[9 * i + k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int g = 3 * i + k;
      double R = F.fab[6 * i + 3 + k];
      if (i + 1 < N) R += F.fab[6 * (i + 1) + k];
      const double rz = F.cn[g] - (k < 2 ? mt : mr) * F.four_dt2 * F.chi[g] - R;
      F.rz[g] = rz;
      if (F.y0) F.y0[g] = (float)(k < 2 && F.f ? rz + F.ds * F.f[k * F.fstride + i] : rz);
    }
  }
}

__device__ __forceinline__ Bcr flag_bcr(const Flag& F) { return Bcr{F.mi, F.bm, F.ey, F.N}; }

}  // namespace beam
