// FSI iteration of one time step (Algorithm 2; Eqs. stress2 and dtheta2) in double precision, as one
// cooperative kernel over a fixed set of CTAs.  Every CTA keeps the float inverse X of the small system in
// shared memory and computes every small vector step (P, right-hand side, refinement, dtheta) itself, so
// grid barriers are needed only where a CTA needs matrix rows another CTA produced:
//   A  body points at theta^(k), the hat map P (Eq. weights), rhs = P E0 (C s* + q_inf) - r^c(k)
//      + S^T (r^theta(k) - (2/dt) J^{-1} r^phidot(k))                              [every CTA, all points]
//   B  K = (ds/h^2) P B0 P^T + (2 ds/dt) S^T J^{-1} S  (16 B0 lookups per entry): without flags, entries
//      over all CTAs (the lower triangle mirrored for the dense B0); with flags, K is already assembled by
//      owned rows during A and B does nothing
//   C  f = K^{-1} rhs to double accuracy by iterative refinement: d = X r with the float inverse X,
//      f += d, r = rhs - K f in double, until |d| <= 1e-10 |f|.  d and f are computed in full by every
//      CTA; each CTA computes the residual rows it owns.  X is carried across iterations and steps and
//      refreshed for each new K by two Newton-Schulz steps X <- 2X - (X K) X (each squares the error
//      I - K X), the products split by owned columns of X K and owned rows of the new X.  It is rebuilt
//      from scratch (blocked float Cholesky and triangular inverse in CTA 0, then W^T W over all CTAs) at
//      the first step, when refinement stalls, or when it diverges.
//   D  dtheta = J^{-1}(r^phidot(k) + ds S f), convergence on max |dtheta| (every CTA computes the same
//      value in the same order, so all CTAs take the same branch without another barrier)
// repeated until max |dtheta| <= tol, then the Newmark update and force outputs (CTA 0).
// Deformable bodies (beam.cuh): during A, warps 4-7 of every CTA build J_d(chi^(k)) and r^zeta(k) of each
// flag, factor J_d and solve for y = J_d^-1 (r^zeta(k) + ds T^T f_prev) (f_prev: the last surface stress)
// and for the columns T J_d^-1 T^T e_r of the rows r the CTA owns.  Meanwhile warps 0-3, once every CTA's
// warps 0-3 have published their points (a barrier of their own), assemble the CTA's owned rows of
// (ds/h^2) P B0 P^T; the CTA then adds to entry (r, c) of its rows the flags' term (2 ds/dt) T J_d^-1 T^T
// from its own column r and publishes the rows before the grid barrier that ends A.  K is then symmetric
// only to the rounding of those FP32 columns and of the two summation orders of (r, c) and (c, r).  After
// the A barrier every CTA subtracts T((2/dt)(chi^(k) + y) - r^chi) from the right-hand side; C starts from
// f_prev with the residual rows rhs + (2 ds/dt) T J_d^-1 T^T f_prev - K f_prev (the same system as
// Eq. stress2, in a form whose FP32 structural solves act on vanishing residuals); D solves
// dchi = J_d^-1 (r^zeta(k) + ds T^T f) (Eq. dchi2) and the convergence test takes max |dchi| as well.
// Data written by other CTAs inside this kernel is read with __ldcg (L2), so no stale L1 line is used.
#include <cooperative_groups.h>
#include <cmath>
#include <climits>
#include <cstring>
#include "beam.cuh"
#include "internal.h"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kMaxSolves = 12;        // refinement solves per attempt
constexpr double kStaleRatio = 0.02;  // |d_s| / |d_{s-1}| above this -> rebuild Kinv for the next iteration
constexpr double kRefineTol = 1e-10;  // stop at |d| <= 1e-10 |f|; the next correction would be ~ratio times that
constexpr int kNsSteps = 2;  // Newton-Schulz steps per refresh of the inverse
constexpr double kNsTrigger = 0.01;  // refinement contraction |d_s| / |d_{s-1}| above this -> refresh X
constexpr int BS = 32;       // Cholesky / inverse / GEMM tile (one warp wide)
constexpr int kMaxBodies = 64;
constexpr int kMaxR = 4;     // rows (and columns) of the small system owned by one CTA
constexpr int kMaxRhs = 1 + kMaxR;  // structural solves per flag in phase A: y and the owned columns
// The distributed variant (nf too large for the float inverse in shared memory): rows per CTA and Newton-Schulz
// steps of a rebuild from a scaled identity.
constexpr int kMaxRB = 12;
constexpr int kNsRebuild = 30;
// Refreshes (one Newton-Schulz step each) per solve attempt of the distributed variant: when one step leaves the
// contraction above the trigger (a body moved far since X was last refreshed), a second or third squares the
// error again; a rebuild from a scaled identity (kNsRebuild steps) is left for an inverse that diverged or an
// attempt that did not converge.
constexpr int kMaxRefreshB = 3;

constexpr unsigned FULL = 0xffffffffu;

struct FsiArgs {
  const void* s0;
  int fp64;
  long ps;
  double x0, y0, h, dt, ds, U, V, tol;
  double two_dt, four_dt2;  // 2/dt and 4/dt^2 (no FP64 divisions per point or entry)
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
  double* rhs;   // [3][nf] residual rows of the refinement (two buffers), right-hand side
  double* K;     // [nf][nf] double, both triangles
  double* f;     // [nf]
  float* Xa;     // [nf][nf] float inverse of K, ping-pong buffer a
  float* Xb;     // [nf][nf] ping-pong buffer b (ctrl[7] says which one is current)
  float* S;      // [nf][nf] float copy of K (Newton-Schulz operand)
  float* T;      // [nf][nf] scratch: X K, or the inverse Cholesky factor during a rebuild
  double* part;  // [2 * gridDim] per-CTA maxima
  unsigned long long* phase_ns;  // [16] accumulated wall time per kernel phase
  int* ctrl;     // [1] iterations of the last step, [2] step index, [4] Kinv valid, [5] solves of the last
                 // step, [6] Kinv rebuilds so far, [7] current X buffer, [8..11] vertex box touched by the
                 // corrector source, [12] Newton-Schulz refreshes in the last step
  int* status;
  double* hist;
  int hist_cap;
  // deformable bodies: free dofs (x, y, theta of nodes 1..n-1) and elements, context-wide numbering
  int n_def, nd_tot, ne_tot, nd_max;
  int nbody_max;  // points of the largest body
  double* bchi;   // [nd_tot] chi_n (updated at the end of the step)
  double* bzeta;  // [nd_tot] zeta_n
  double* bzdot;  // [nd_tot] zetadot_n
  double* bref;   // [ne_tot][3] chord rotation psi and unit chord (c, s) at chi_n
  double* G;      // [nf][nf] column-major: column r = T J_d^-1 T^T e_r for deformable rows r
  // sparse B0' (windowed columns, b0w_lookup) in place of the dense B0, or NULL
  const double* Bw;
  int bw;
  int* pcij;      // [nb][2] hat cell (ci, cj) of every point, for the window lookups
  // prescribed kinematics ([kin_cap][n_bodies][6], slot = step mod kin_cap) or NULL; nkb = n_bodies when set
  const double* kin;
  int kin_cap, nkb;
  // appended points: Omega_0 index of every body point (-1: interpolated by P) and their face windows
  int n_box;
  const int* app_idx;
  const FaceWindow* app_win;
  // bounded wait of the warps 0-3 barrier: poll limit, and arrivals it waits for beyond the grid's (a test
  // sets these to make the wait run out; 0 in normal runs)
  unsigned lb_spins;
  int lb_missing;
  // Omega_0 as a union of boxes (reading R16): n_sdb boxes (grid vertex i_lo, i_hi, j_lo, j_hi) and the
  // Omega_0 index of every vertex of the bounding box (i_lo, j_lo, ni, nj above); n_sdb = 1: one box
  int n_sdb;
  int sdb[16][4];
  const int* sd_map;
  // distributed variant: the correction d = X r of every row, and per-row absolute sums of K (rebuild)
  double* dvec;
  double* rsum;
  float* resf;  // float copies of the residual rows, [2][nf] by solve parity
};

// level-0 streamfunction at vertex offset o: fp64 = 0 float, 1 double, 2 float pair (the mixed mode)
__device__ __forceinline__ double load_s(const FsiArgs& a, long o) {
  if (a.fp64 == 2) return (double)((const f2s*)a.s0)[o];
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

// Wall time per phase of the kernel in nanoseconds (%globaltimer), kept by thread 0 of CTA 0 in shared
// memory and added to the global totals once at the end of the launch.  Phases: 0 A, 1 B, 2 inverse
// refresh, 3 inverse rebuild, 4 refinement solves, 5 double residuals, 6 dtheta/convergence, 7 outputs;
// sub-phases (split of 2, 4 and 5): 8 X K columns, 9 new X rows, 10 reload of X, 11 d = X r,
// 12 residual rows and barrier, 13 residual gather.
constexpr int kPhases = 24;
struct PhaseClock {
  unsigned long long* acc;  // shared [kPhases]
  bool on;
  unsigned long long last, sub_last;
  __device__ static unsigned long long now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
  }
  __device__ PhaseClock(unsigned long long* a, bool o) : acc(a), on(o) {
    if (on) {
      for (int k = 0; k < kPhases; ++k) acc[k] = 0;
      last = sub_last = now();
    }
  }
  __device__ void mark(int phase) {
    if (!on) return;
    const unsigned long long t = now();
    acc[phase] += t - last;
    last = sub_last = t;
  }
  __device__ void sub(int phase) {
    if (!on) return;
    const unsigned long long t = now();
    acc[phase] += t - sub_last;
    sub_last = t;
  }
  __device__ void flush(unsigned long long* global) {
    if (!on || !global) return;
    for (int k = 0; k < kPhases; ++k) global[k] += acc[k];
  }
};

// Deterministic block reductions (fixed tree); all threads must call; result valid in every thread.
// Warp shuffle tree, then warp 0 combines the warp results in warp order and broadcasts: two barriers per
// reduction, FP64 work only in the first step and in warp 0 (FP64 throughput per SM is low on sm_103).
__device__ double block_sum(double x, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  if (lane == 0) red[wid] = x;
  __syncthreads();
  if (wid == 0) {
    double r = red[0];
    for (int w = 1; w < nw; ++w) r += red[w];
    if (lane == 0) red[32] = r;
  }
  __syncthreads();
  return red[32];
}

// Sums over the CTA of K values per thread (nw K + K <= 256): each by warp butterflies, then warp 0 adds the
// warps' partial sums in order; one set of barriers for all K.
template <int K>
__device__ void block_sum_k(double (&x)[K], double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < K; ++k) x[k] += __shfl_xor_sync(FULL, x[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[wid * K + k] = x[k];
  __syncthreads();
  if (wid == 0 && lane < K) {
    double r = red[lane];
    for (int w = 1; w < nw; ++w) r += red[w * K + lane];
    red[nw * K + lane] = r;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) x[k] = red[nw * K + k];
  __syncthreads();  // red is free again
}

__device__ double block_max(double x, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(FULL, x, o));
  if (lane == 0) red[wid] = x;
  __syncthreads();
  if (wid == 0) {
    double r = red[0];
    for (int w = 1; w < nw; ++w) r = fmax(r, red[w]);
    if (lane == 0) red[32] = r;
  }
  __syncthreads();
  return red[32];
}

// Block-wide maxima of two non-negative floats given as bit patterns (integer order = float order; +inf
// and NaN patterns sort above every finite value).  One barrier pair.
// dst[k] = src[k], k < n (global, written in this launch), by the CTA: a thread's loads issued together
__device__ __forceinline__ void gather_f(float* dst, const float* src, int n) {
  for (int k0 = threadIdx.x; k0 < n; k0 += blockDim.x * 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = k0 + u * (int)blockDim.x < n ? __ldcg(&src[k0 + u * blockDim.x]) : 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u * (int)blockDim.x < n) dst[k0 + u * blockDim.x] = v[u];
  }
}

// block maxima of two 64-bit patterns (non-negative doubles order as their bit patterns); red: >= 64 doubles
__device__ void block_max2_bits64(unsigned long long& a, unsigned long long& b, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = max(a, __shfl_xor_sync(FULL, a, o));
    b = max(b, __shfl_xor_sync(FULL, b, o));
  }
  unsigned long long* r = reinterpret_cast<unsigned long long*>(red);
  if (lane == 0) {
    r[wid] = a;
    r[32 + wid] = b;
  }
  __syncthreads();
  unsigned long long ra = r[0], rb = r[32];
  for (int w = 1; w < nw; ++w) {
    ra = max(ra, r[w]);
    rb = max(rb, r[32 + w]);
  }
  __syncthreads();
  a = ra;
  b = rb;
}

__device__ void block_max2_bits(unsigned& a, unsigned& b, unsigned* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = __reduce_max_sync(FULL, a);
  b = __reduce_max_sync(FULL, b);
  if (lane == 0) {
    red[wid] = a;
    red[32 + wid] = b;
  }
  __syncthreads();
  unsigned ra = red[0], rb = red[32];
  for (int w = 1; w < nw; ++w) {
    ra = max(ra, red[w]);
    rb = max(rb, red[32 + w]);
  }
  __syncthreads();
  a = ra;
  b = rb;
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

// Shared-memory layout of the kernel (byte offsets, 16-byte aligned): X (or the Cholesky factor in CTA 0
// during a rebuild), owned K rows, the vectors rhs, f, r, the hat weights, a float4 work row, hat indices;
// for deformable bodies the iterate chi^(k), r^zeta(k), the step constants r^zeta_n and r^chi_n, the
// reference chords, the element end forces, the factor blocks of J_d
// (Mi, Bm, and per flag [Em | y] where the element tangents are staged before the factorization) and the
// right-hand sides of the structural solves.
struct FsiLayout {
  size_t xs, krow, vec, pw, work, rf, pidx, pcij, pbody, tors, torsf;
  size_t chi, rz, cn, rchi, ref, fab, mi, bm, ey, ys, kb;
  size_t total;
};
struct BeamDims {
  int nd, ne, nd_max;  // free dofs and elements of all flags, dofs of the largest flag
  int nkb;             // bodies with a per-step kinematics block (all bodies when a driven plate exists)
  int nbody_max;       // points of the largest body (the distributed variant's copy of X's owned blocks)
};
__host__ __device__ inline size_t al16(size_t b) { return (b + 15) / 16 * 16; }
// Work area of the distributed variant (floats): a 64 x 33 + 32 x 64 tile of the block products, or the
// owned rows' blocks of X (kMaxRB rows of 2 nbody_max floats)
__host__ __device__ inline size_t fsi_big_work_floats(int nbody_max) {
  const size_t t = 64 * 33 + 32 * 64, x = (size_t)kMaxRB * 2 * (size_t)nbody_max;
  return t > x ? t : x;
}
// Row stride (floats) of the float matrices X, X K and K in global and shared memory: a multiple of 4 (rows
// start on 16 bytes) with an odd number of 16-byte units, so that threads reading consecutive rows with
// 128-bit loads hit distinct banks.  Columns nf .. ldx-1 stay zero.
__host__ __device__ inline int fsi_ldx(int nf) {
  int l = (nf + 3) / 4 * 4;
  if (((l / 4) & 1) == 0) l += 4;
  return l;
}
// big: the distributed variant, which keeps X and K in global memory (no X or owned K rows in shared memory;
// the work area holds the tiles of its block products).
__host__ __device__ inline FsiLayout fsi_layout(int nf, int nb, BeamDims bd, bool big = false) {
  FsiLayout L;
  const size_t lx = (size_t)fsi_ldx(nf);
  const size_t xa = (size_t)nf * lx, xb = (size_t)nf * (size_t)(nf | 1);  // X, or the Cholesky factor
  L.xs = 0;
  L.krow = L.xs + (big ? 0 : al16((xa > xb ? xa : xb) * 4));
  L.vec = L.krow + (big ? 0 : al16((size_t)kMaxR * nf * 8));
  L.pw = L.vec + al16((size_t)3 * nf * 8);
  L.work = L.pw + al16((size_t)4 * nb * 8);
  // big: the tiles of the block products, or between two changes of X the CTA's owned rows of X's blocks
  L.rf = L.work + (big ? al16(fsi_big_work_floats(bd.nbody_max) * 4) : al16(lx * 16));
  L.pidx = L.rf + al16(lx * 4);
  L.pcij = L.pidx + al16((size_t)4 * nb * 4);
  L.pbody = L.pcij + al16((size_t)2 * nb * 4);
  L.tors = L.pbody + al16((size_t)nb * 4);
  L.torsf = L.tors + (big ? al16((size_t)nf * 8) : 0);
  L.chi = L.torsf + (big ? al16((size_t)nf * 4) : 0);
  L.rz = L.chi + al16((size_t)bd.nd * 8);
  L.cn = L.rz + al16((size_t)bd.nd * 8);
  L.rchi = L.cn + al16((size_t)bd.nd * 8);
  L.ref = L.rchi + al16((size_t)bd.nd * 8);
  L.fab = L.ref + al16((size_t)3 * bd.ne * 8);
  L.mi = L.fab + al16((size_t)6 * bd.ne * 8);
  L.bm = L.mi + al16((size_t)6 * bd.ne * 4);
  L.ey = L.bm + al16((size_t)9 * bd.ne * 4);
  L.ys = L.ey + al16((size_t)12 * bd.ne * 4);
  L.kb = L.ys + al16((size_t)(big ? 1 + kMaxRB : kMaxRhs) * bd.nd_max * 4);
  L.total = L.kb + al16((size_t)bd.nkb * KB_N * 8);
  return L;
}

// Xs <- the nf x ldx float matrix src by bulk asynchronous copies (thread 0 issues, every thread waits).
// The caller guarantees that no thread still reads Xs.  A copy that does not land within the wait limit
// records FSI_ERR_TIMEOUT.
__device__ void load_x(float* Xs, const float* src, int nf, int ldx, uint64_t* bar, uint32_t* phase, int* status) {
  const uint32_t bytes = (uint32_t)nf * (uint32_t)ldx * 4u;
  if (threadIdx.x == 0) {
    tc::fence_proxy_async_all();
    tc::mbar_arrive_expect_tx(bar, bytes);
    const uint32_t chunk = 32768u;
    for (uint32_t o = 0; o < bytes; o += chunk) {
      const uint32_t n = bytes - o < chunk ? bytes - o : chunk;
      tc::bulk_g2s(reinterpret_cast<char*>(Xs) + o, reinterpret_cast<const char*>(src) + o, n, bar);
    }
  }
  if (!tc::mbar_wait(bar, *phase, 2000000000ull)) dev_set_status(status, FSI_ERR_TIMEOUT);
  *phase ^= 1u;
}

// Barrier of warps 4-7 only (named barrier 1), used while warps 0-3 work on the body points.
__device__ __forceinline__ void named_sync_upper() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Barrier of warps 0-3 only (named barrier 2), used while warps 4-7 work on the flags.
__device__ __forceinline__ void named_sync_lower() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

// Barrier of warps 0-3 of every CTA while warps 4-7 still work on the flags: named barrier 2 inside the CTA,
// an arrival counter in global memory across CTAs (all CTAs of the cooperative launch are resident).  The
// counter grows by gridDim.x per use (target = uses so far * gridDim.x) and CTA 0 resets it at the end of
// the launch.  A wait that does not end within the limit records FSI_ERR_TIMEOUT and goes on, so that every
// CTA keeps to the same sequence of barriers.
// spin_limit bounds the wait (polls of about 64 ns each); a test may lower it and add arrivals that never
// come, so that the wait runs out (the failure-detection path, with no copies in flight).
__device__ void lower_grid_barrier(int* cnt, int target, int* status, unsigned spin_limit) {
  named_sync_lower();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(cnt, 1);
    unsigned spins = 0;
    while (*(volatile int*)cnt < target) {
      if (++spins > spin_limit) {
        dev_set_status(status, FSI_ERR_TIMEOUT);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  named_sync_lower();
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// ---- Distributed small-system solver (the kernel's BIG variant) -------------------------------------------
// X is a block-Jacobi float inverse of K: one block per body (its 2n rows and columns, x then y components),
// kept in global memory with K's float copy S.  Row r of the block of body b has its columns at
// off + t (t < n) and nb + off + t - n (n <= t < 2n).  A CTA owns rows r0 .. r0 + nr - 1 of every matrix;
// consecutive owned rows with the same block form a group, whose rows are multiplied together so that each
// CTA reads the block operand once per product.  X is refreshed by one Newton-Schulz step when the refinement
// contracts by more than 0.05 per solve, up to kMaxRefreshB times per solve attempt, and rebuilt from a scaled
// identity only when it diverged or an attempt did not converge.
struct RowBlock {
  int off, n;
};
__device__ __forceinline__ RowBlock row_block(const FsiArgs& a, int r) {
  const BodyDev& b = a.bodies[a.point_body[r % a.nb]];
  return RowBlock{b.off, b.n};
}
__device__ __forceinline__ int blk_col(RowBlock b, int nb, int t) { return t < b.n ? b.off + t : nb + b.off + (t - b.n); }

// Tiled block products of the Newton-Schulz steps: out = alpha X0 + beta A B on every block (A, B, X0, out
// restricted to the block's rows and columns), each block's output cut into 64 x 64 tiles and all tiles of
// all blocks dealt round-robin to the CTAs.  A CTA streams a tile's 64 rows of A and 64 columns of B through
// shared memory in steps of 32 (the next step's loads issued before the current step is multiplied); a
// thread accumulates a 4 x 4 part of the tile.  smem: 64 x 33 + 32 x 64 floats.
constexpr int kGT = 64, kGK = 32;
__device__ void blk_gemm(const FsiArgs& a, const float* A, const float* B, const float* X0, float alpha, float beta,
                         float* out, int lx, float* smem) {
  const int tid = threadIdx.x, nb = a.nb;
  const int ty = tid >> 4, tx = tid & 15;  // rows 4 ty .. 4 ty + 3, columns 4 tx .. 4 tx + 3 of the tile
  float* As = smem;                        // [kGT][kGK + 1]
  float* Bs = smem + kGT * (kGK + 1);      // [kGK][kGT]
  int tiles_before = 0;
  for (int bi = 0; bi < a.n_bodies; ++bi) {
    const BodyDev bd = a.bodies[bi];
    const RowBlock b{bd.off, bd.n};
    const int n2 = 2 * b.n, nt = (n2 + kGT - 1) / kGT;
    for (int tile = (int)blockIdx.x - tiles_before % (int)gridDim.x; tile < nt * nt; tile += gridDim.x) {
      if (tile < 0) continue;
      const int i0 = (tile / nt) * kGT, j0 = (tile % nt) * kGT;
      float acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
      float ra[8], rb[8];  // this thread's share of the next step's A (64 x 32) and B (32 x 64) tiles
      auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = tid + q * 256;
          const int ar = e >> 5, ak = e & 31;  // A tile: row ar, step column ak
          const int gi = i0 + ar, gk = k0 + ak;
          ra[q] = (gi < n2 && gk < n2) ? __ldcg(&A[(long)blk_col(b, nb, gi) * lx + blk_col(b, nb, gk)]) : 0.0f;
          const int bk = e >> 6, bc = e & 63;  // B tile: step row bk, column bc
          const int gk2 = k0 + bk, gj = j0 + bc;
          rb[q] = (gk2 < n2 && gj < n2) ? __ldcg(&B[(long)blk_col(b, nb, gk2) * lx + blk_col(b, nb, gj)]) : 0.0f;
        }
      };
      load(0);
      for (int k0 = 0; k0 < n2; k0 += kGK) {
        __syncthreads();  // the previous step's tiles are no longer read
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = tid + q * 256;
          As[(e >> 5) * (kGK + 1) + (e & 31)] = ra[q];
          Bs[e] = rb[q];
        }
        __syncthreads();
        if (k0 + kGK < n2) load(k0 + kGK);  // in flight while this step is multiplied
#pragma unroll 8
        for (int kk = 0; kk < kGK; ++kk) {
          float av[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) av[u] = As[(4 * ty + u) * (kGK + 1) + kk];
          const float4 b4 = reinterpret_cast<const float4*>(Bs)[kk * (kGT / 4) + tx];  // 16-byte aligned rows
          const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int gi = i0 + 4 * ty + u;
        if (gi >= n2) continue;
        const long ro = (long)blk_col(b, nb, gi) * lx;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int gj = j0 + 4 * tx + v;
          if (gj >= n2) continue;
          const long o = ro + blk_col(b, nb, gj);
          out[o] = alpha != 0.0f ? alpha * __ldcg(&X0[o]) + beta * acc[u][v] : beta * acc[u][v];
        }
      }
    }
    tiles_before += nt * nt;
  }
  __syncthreads();
}

template <bool BIG>
__global__ void __launch_bounds__(256, 1) k_fsi(FsiArgs a) {
  constexpr int MR = BIG ? kMaxRB : kMaxR;  // owned rows per CTA
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ double red[256];
  __shared__ unsigned redu[64];
  __shared__ double b_th[kMaxBodies], b_ph[kMaxBodies], b_rphi[kMaxBodies], b_rth[kMaxBodies], b_jac[kMaxBodies];
  __shared__ double b_tp[kMaxBodies];  // angle of the iterate that produced the current f (S, P of the solve)
  __shared__ double b_sn[kMaxBodies], b_cs[kMaxBodies];  // sin, cos of theta0 + theta^(k)
  __shared__ double b_ijac[kMaxBodies], b_kc[kMaxBodies];  // 1/J and (2 ds/dt)/J
  __shared__ int bt_s[kMaxBodies], boff_s[kMaxBodies];     // type and first point of every body
  __shared__ int bn_s[kMaxBodies];                          // points of every body
  __shared__ int bbx_s[kMaxBodies][4];  // hat-cell box of every body at the iterate: i_min, i_max, j_min, j_max
  __shared__ int sh_bad;
  __shared__ unsigned long long sh_phase[kPhases];
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
  const long gtid = (long)blockIdx.x * nthr + tid;
  const long gsize = (long)gridDim.x * nthr;
  const long wg = gtid >> 5, nwg = gsize >> 5;
  const int nb = a.nb, nf = a.nf;
  const int ld = nf | 1;        // row stride of the Cholesky factor during a rebuild
  const int lx = fsi_ldx(nf);   // row stride of X, X K and the float K
  const double dt = a.dt;
  // residual rows published to the other CTAs, double-buffered by solve parity: a CTA may write the rows of
  // solve s+1 while another is still reading those of solve s (one barrier per solve)
  double* const res0 = a.rhs;
  double* const res1 = a.rhs + nf;
  // rows (and columns) of the small system owned by this CTA: [r0, r0 + nr)
  const int R = (nf + (int)gridDim.x - 1) / (int)gridDim.x;
  const int r0 = min(nf, (int)blockIdx.x * R);
  const int nr = min(nf, r0 + R) - r0;
  const FsiLayout L = fsi_layout(nf, nb, BeamDims{a.nd_tot, a.ne_tot, a.nd_max, a.nkb, a.nbody_max}, BIG);
  float* Xs = reinterpret_cast<float*>(dyn_smem + L.xs);
  double* Krow = reinterpret_cast<double*>(dyn_smem + L.krow);
  double* rhs_s = reinterpret_cast<double*>(dyn_smem + L.vec);
  double* f_s = rhs_s + nf;
  double* r_s = f_s + nf;
  double* pw_s = reinterpret_cast<double*>(dyn_smem + L.pw);
  float4* work4 = reinterpret_cast<float4*>(dyn_smem + L.work);
  float* rf = reinterpret_cast<float*>(dyn_smem + L.rf);  // float copy of the vector X is applied to
  int* pidx_s = reinterpret_cast<int*>(dyn_smem + L.pidx);
  int* pcij_s = reinterpret_cast<int*>(dyn_smem + L.pcij);
  int* pb_s = reinterpret_cast<int*>(dyn_smem + L.pbody);  // body of every point
  // BIG: the torsional moment arm of every unknown at the iterate, (p - off) ds (-sin, cos)[component]
  double* tors_s = reinterpret_cast<double*>(dyn_smem + L.tors);
  float* torsf_s = reinterpret_cast<float*>(dyn_smem + L.torsf);  // BIG: its float copy
  double* chi_s = reinterpret_cast<double*>(dyn_smem + L.chi);  // chi^(k) of every flag
  double* rz_s = reinterpret_cast<double*>(dyn_smem + L.rz);    // r^zeta(k)
  double* cn_s = reinterpret_cast<double*>(dyn_smem + L.cn);      // r^zeta_n of every free dof
  double* rchi_s = reinterpret_cast<double*>(dyn_smem + L.rchi);  // r^chi_n = (2/dt) chi_n + zeta_n
  double* ref_s = reinterpret_cast<double*>(dyn_smem + L.ref);    // reference chords [ne][3]
  double* fab_s = reinterpret_cast<double*>(dyn_smem + L.fab);  // element end forces [ne][6]
  float* mi_s = reinterpret_cast<float*>(dyn_smem + L.mi);
  float* bm_s = reinterpret_cast<float*>(dyn_smem + L.bm);
  float* ey_s = reinterpret_cast<float*>(dyn_smem + L.ey);
  float* ys_s = reinterpret_cast<float*>(dyn_smem + L.ys);
  // per-body kinematics block of this step (KB_* in internal.h), NULL without driven bodies
  double* kb_s = a.nkb > 0 ? reinterpret_cast<double*>(dyn_smem + L.kb) : nullptr;
  float* tile = reinterpret_cast<float*>(dyn_smem + L.work);  // BIG: tile of the block products
  // BIG: the owned rows in groups of consecutive rows with the same block (same in every thread of the CTA)
  auto for_groups = [&](auto fn) {
    int g0 = r0;
    while (g0 < r0 + nr) {
      const RowBlock b = row_block(a, g0);
      int g1 = g0 + 1;
      while (g1 < r0 + nr && row_block(a, g1).off == b.off) ++g1;
      fn(g0, g1 - g0, b);
      g0 = g1;
    }
  };
  // rows owned by this CTA that are x / y rows of a free flag node: their structural column is solved here
  __shared__ int g_body[MR], g_dof[MR];
  if (tid < MR) {
    g_body[tid] = -1;
    g_dof[tid] = 0;
    if (tid < nr && a.n_def > 0) {
      const int r = r0 + tid, ca = r / nb, p = r % nb;
      const int bi = a.point_body[p];
      const BodyDev b = a.bodies[bi];
      if (b.type == FSI_BODY_DEFORMABLE && p > b.off) {
        g_body[tid] = bi;
        g_dof[tid] = 3 * (p - b.off - 1) + ca;
      }
    }
  }
  for (int p = tid; p < nb; p += nthr) pb_s[p] = a.point_body[p];
  for (int bi = tid; bi < a.n_bodies; bi += nthr) {
    bt_s[bi] = a.bodies[bi].type;
    boff_s[bi] = a.bodies[bi].off;
    bn_s[bi] = a.bodies[bi].n;
  }
  for (int g = tid; g < a.nd_tot; g += nthr) chi_s[g] = a.bchi[g];
  for (int e = tid; e < 3 * a.ne_tot; e += nthr) ref_s[e] = a.bref[e];
  for (int bi = 0; bi < a.n_bodies && a.n_def > 0; ++bi) {  // step constants of App. A, FP64
    const BodyDev b = a.bodies[bi];
    if (b.type != FSI_BODY_DEFORMABLE) continue;
    const int N = b.n - 1, d0 = 3 * b.el_off;
    for (int q = tid; q < 3 * N; q += nthr) {
      const int g = d0 + q;
      cn_s[g] = beam::node_mass(b.mu, a.ds, N, q / 3, q % 3) *
                (a.four_dt2 * a.bchi[g] + 2.0 * a.two_dt * a.bzeta[g] + a.bzdot[g]);
      rchi_s[g] = a.two_dt * a.bchi[g] + a.bzeta[g];
    }
  }
  // with flags the small system is solved for the correction to the previous surface stress f_prev (the
  // last iterate, or the last step's f): see the refinement below
  if (a.n_def > 0)
    for (int k = tid; k < nf; k += nthr) f_s[k] = a.f[k];

  // per-CTA copy of the structural state (identical in every CTA)
  for (int bi = tid; bi < a.n_bodies; bi += nthr) {
    const BodyDev b = a.bodies[bi];
    const BodyState s = a.st[bi];
    if (b.type == FSI_BODY_TORSIONAL) {
      b_jac[bi] = 4.0 * b.inertia / (dt * dt) + 2.0 * b.damping / dt + b.stiffness;
      b_rphi[bi] = b.inertia * (4.0 * s.theta / (dt * dt) + 4.0 * s.phi / dt + s.phidot) +
                   b.damping * (2.0 * s.theta / dt + s.phi);
      b_rth[bi] = s.phi + 2.0 / dt * s.theta;
      b_ijac[bi] = 1.0 / b_jac[bi];
      b_kc[bi] = (2.0 * a.ds / dt) / b_jac[bi];
      b_th[bi] = s.theta;
      b_ph[bi] = s.phi;
      b_tp[bi] = s.theta;
    } else {
      b_jac[bi] = b_ijac[bi] = 1.0;
      b_kc[bi] = 0.0;
      b_rphi[bi] = b_rth[bi] = b_th[bi] = b_ph[bi] = b_tp[bi] = 0.0;
    }
    if (kb_s) {  // prescribed kinematics at the end of this step (Sec. 5.1, Eq. newtonseldg)
      const BodyDev b = a.bodies[bi];
      double* k = kb_s + bi * KB_N;
      for (int m = 0; m < KB_N; ++m) k[m] = 0.0;
      const int src = b.type == FSI_BODY_DRIVEN ? bi : (b.type == FSI_BODY_TORSIONAL ? b.driver : -1);
      k[KB_X] = b.hx;
      k[KB_Y] = b.hy;
      k[KB_T0] = b.theta0;
      if (src >= 0) {
        const double* q = a.kin + ((long)(a.ctrl[2] % a.kin_cap) * a.n_bodies + src) * 6;
        double sa, ca;
        sincos(q[3], &sa, &ca);
        if (b.type == FSI_BODY_DRIVEN) {  // reference point, its velocity, plate direction (sin, -cos)(alpha1)
          k[KB_X] = b.hx + q[0];
          k[KB_VX] = q[1];
          k[KB_SA] = sa;
          k[KB_CA] = ca;
          k[KB_AD] = q[4];
        } else {  // hinge at l1 along the driven plate, its velocity, rest direction alpha1 - pi/2, g terms
          const BodyDev d = a.bodies[src];
          k[KB_X] = d.hx + q[0] + b.l1 * sa;
          k[KB_Y] = d.hy - b.l1 * ca;
          k[KB_VX] = q[1] + b.l1 * q[4] * ca;
          k[KB_VY] = b.l1 * q[4] * sa;
          k[KB_AD] = q[4];
          k[KB_T0] = q[3] - 0.5 * M_PI;
          const double ml = b.mass * b.l1 * b.l2;
          k[KB_GX] = -b.mass * b.l2 * q[2];
          k[KB_GI] = -b.inertia * q[5];
          k[KB_GC] = -ml * q[5];
          k[KB_GS] = -ml * q[4] * q[4];
        }
      }
    }
  }
  int kinv_valid = *(volatile int*)&a.ctrl[4];
  int cur = *(volatile int*)&a.ctrl[7];
  // BIG: changes of X in this launch, and the change whose owned-row blocks the tile area holds (-1: none)
  int x_version = 0, xs_version = -1;
  __shared__ uint64_t xbar;  // bulk copies of X into shared memory
  uint32_t xphase = 0;
  if (tid == 0) {
    tc::mbar_init(&xbar, 1);
    tc::fence_mbar_init();
  }
  for (int k = nf + tid; k < lx; k += nthr) rf[k] = 0.0f;
  __syncthreads();
  if (!BIG && kinv_valid) load_x(Xs, cur ? a.Xb : a.Xa, nf, lx, &xbar, &xphase, a.status);
  PhaseClock clk(sh_phase, blockIdx.x == 0 && tid == 0 && a.phase_ns);
  __syncthreads();

  // Entry (r, c) of K = (ds/h^2) P B0 P^T + (2 ds/dt) S^T J^{-1} S; with_g = false leaves out the flags'
  // (2 ds/dt) T J_d^-1 T^T.
  const bool dense = a.Bw == nullptr;
  // The windowed B0': hat cells of points pa and pb more than bw + 1 cells apart share no entry of the window,
  // and for nearer ones sum_{al, be} w_al(pa) w_be(pb) B0'[(ca, vertex al)][(cb, vertex be)] comes from the
  // windows of pb's hat vertices (its sixteen loads independent: all issued before the sums).
  auto window_near = [&](int dj0, int di0) -> bool {
    return dj0 <= a.bw + 1 && dj0 >= -a.bw - 1 && di0 <= a.bw + 1 && di0 >= -a.bw - 1;
  };
  auto window_acc = [&](int pa, int ca, int pb, int cb, int dj0, int di0) -> double {
    const int bw = a.bw, side = 2 * bw + 1;
    const long carea = (long)side * side;
    int ib[4];
    double wb[4], t[4];
#pragma unroll
    for (int be = 0; be < 4; ++be) {
      ib[be] = pidx_s[4 * pb + be];
      wb[be] = pw_s[4 * pb + be];
    }
#pragma unroll
    for (int al = 0; al < 4; ++al) {
      t[al] = 0.0;
#pragma unroll
      for (int be = 0; be < 4; ++be) {
        const int dj = dj0 + (al >> 1) - (be >> 1), di = di0 + (al & 1) - (be & 1);
        if (dj >= -bw && dj <= bw && di >= -bw && di <= bw)
          t[al] += wb[be] * a.Bw[((long)cb * a.n_sd + ib[be]) * 2 * carea + (long)ca * carea + (long)(dj + bw) * side +
                                 (di + bw)];
      }
    }
    double acc = 0.0;
#pragma unroll
    for (int al = 0; al < 4; ++al) acc += pw_s[4 * pa + al] * t[al];
    return acc;
  };
  // window_acc in two halves, so that a thread can issue the loads of several entries before it sums any:
  // v[4 al + be] = B0'[(ca, vertex al of pa)][(cb, vertex be of pb)] where the pair lies in the window (zero
  // elsewhere, or everywhere when on is false); window_sum then adds exactly the terms window_acc adds, in its
  // order, so the two give the same bits
  auto window_load = [&](int ca, int pb, int cb, int dj0, int di0, bool on, double* v) {
    const int bw = a.bw, side = 2 * bw + 1;
    const long carea = (long)side * side;
#pragma unroll
    for (int be = 0; be < 4; ++be) {
      const long col = ((long)cb * a.n_sd + (on ? pidx_s[4 * pb + be] : 0)) * 2 * carea + (long)ca * carea;
#pragma unroll
      for (int al = 0; al < 4; ++al) {
        const int dj = dj0 + (al >> 1) - (be >> 1), di = di0 + (al & 1) - (be & 1);
        const bool in = on && dj >= -bw && dj <= bw && di >= -bw && di <= bw;
        v[4 * al + be] = in ? a.Bw[col + (long)(dj + bw) * side + (di + bw)] : 0.0;
      }
    }
  };
  auto window_sum = [&](int pa, int pb, int dj0, int di0, const double* v) -> double {
    const int bw = a.bw;
    double wb[4], acc = 0.0;
#pragma unroll
    for (int be = 0; be < 4; ++be) wb[be] = pw_s[4 * pb + be];
#pragma unroll
    for (int al = 0; al < 4; ++al) {
      double t = 0.0;
#pragma unroll
      for (int be = 0; be < 4; ++be) {
        const int dj = dj0 + (al >> 1) - (be >> 1), di = di0 + (al & 1) - (be & 1);
        if (dj >= -bw && dj <= bw && di >= -bw && di <= bw) t += wb[be] * v[4 * al + be];
      }
      acc += pw_s[4 * pa + al] * t;
    }
    return acc;
  };
  // fluid_only: the sum over the hat vertices alone, without the factor ds/h^2 and the structural terms
  auto k_entry = [&](int r, int cidx, bool with_g, bool fluid_only = false) -> double {
    const double kscale = a.ds / (a.h * a.h);
    const long n2 = 2L * a.n_sd;
    const int ca = r / nb, pa = r % nb, cb = cidx / nb, pb = cidx % nb;
    double acc = 0.0;
    int ib[4];
    double wb[4];
#pragma unroll
    for (int be = 0; be < 4; ++be) {
      ib[be] = pidx_s[4 * pb + be];
      wb[be] = pw_s[4 * pb + be];
    }
    if (dense) {
      for (int al = 0; al < 4; ++al) {
        const long row = (long)ca * a.n_sd + pidx_s[4 * pa + al];
        const double wa = pw_s[4 * pa + al];
        const double* brow = a.B0 + row * n2 + (long)cb * a.n_sd;
        double t = 0.0;
#pragma unroll
        for (int be = 0; be < 4; ++be) t += wb[be] * brow[ib[be]];
        acc += wa * t;
      }
    } else {  // B0'[(ca, vertex al of pa)][(cb, vertex be of pb)] from the column's window
      const int dj0 = pcij_s[2 * pa + 1] - pcij_s[2 * pb + 1], di0 = pcij_s[2 * pa] - pcij_s[2 * pb];
      // every vertex pair lies outside the window when the hat cells are more than bw + 1 apart
      if (window_near(dj0, di0)) acc = window_acc(pa, ca, pb, cb, dj0, di0);
    }
    if (fluid_only) return acc;
    double kv = kscale * acc;
    const int ba = pb_s[pa], bbd = pb_s[pb];
    if (ba == bbd && bt_s[ba] == FSI_BODY_TORSIONAL) {
      const double sn = b_sn[ba], cs = b_cs[ba];
      const double sa = (double)(pa - boff_s[ba]) * a.ds * (ca == 0 ? -sn : cs);
      const double sb = (double)(pb - boff_s[ba]) * a.ds * (cb == 0 ? -sn : cs);
      kv += b_kc[ba] * sa * sb;
    } else if (with_g && ba == bbd && bt_s[ba] == FSI_BODY_DEFORMABLE) {
      // (2 ds/dt) T J_d^-1 T^T, symmetric: the entry of the lower triangle (column min(r, c))
      kv += a.ds * a.two_dt * __ldcg(&a.G[cidx <= r ? (long)cidx * nf + r : (long)r * nf + cidx]);
    }
    return kv;
  };
  // Bodies ba and bb can have non-zero entries between them in K: always with the dense B0 (and for a body
  // with itself); with the windowed B0' only when their hat-cell boxes come within the window (bw + 1 cells),
  // since every entry of two points farther apart is dropped.  K keeps exact zeros elsewhere, so sums over
  // the coupled columns alone give the same bits as over all columns.
  auto couples = [&](int ba, int bb) -> bool {
    if (dense || ba == bb) return true;
    const int gi = max(bbx_s[ba][0] - bbx_s[bb][1], bbx_s[bb][0] - bbx_s[ba][1]);
    const int gj = max(bbx_s[ba][2] - bbx_s[bb][3], bbx_s[bb][2] - bbx_s[ba][3]);
    return gi <= a.bw + 1 && gj <= a.bw + 1;
  };
  // (K f)_r by a warp over the columns of the bodies that couple with row r's body (the other blocks of K are
  // zero): two chains per lane, summed in a fixed order
  auto coupled_dot = [&](int r) -> double {
    const int ba = pb_s[r % nb];
    const double* kr = a.K + (long)r * nf;
    double c0 = 0.0, c1 = 0.0;
    for (int bb = 0; bb < a.n_bodies; ++bb) {
      if (!couples(ba, bb)) continue;
      const int n = bn_s[bb];
      for (int comp = 0; comp < 2; ++comp) {
        const int off = comp * nb + boff_s[bb];
        for (int t0 = lane; t0 < n; t0 += 32 * 8) {  // the lane's loads of a segment issued together
          double kv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int t = t0 + 32 * u;
            kv[u] = t < n ? __ldcg(&kr[off + t]) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 8; u += 2) {
            const int t = t0 + 32 * u;
            if (t < n) c0 += kv[u] * f_s[off + t];
            if (t + 32 < n) c1 += kv[u + 1] * f_s[off + t + 32];
          }
        }
      }
    }
    return c0 + c1;
  };
  // hat-cell boxes of the bodies from pcij_s, by nt threads of index tl with their own barrier
  auto body_boxes = [&](int tl, int nt, auto sync) {
    for (int bi = tl; bi < a.n_bodies; bi += nt) {
      bbx_s[bi][0] = bbx_s[bi][2] = INT_MAX;
      bbx_s[bi][1] = bbx_s[bi][3] = INT_MIN;
    }
    sync();
    for (int p = tl; p < nb; p += nt) {
      const int bi = pb_s[p];
      atomicMin(&bbx_s[bi][0], pcij_s[2 * p]);
      atomicMax(&bbx_s[bi][1], pcij_s[2 * p]);
      atomicMin(&bbx_s[bi][2], pcij_s[2 * p + 1]);
      atomicMax(&bbx_s[bi][3], pcij_s[2 * p + 1]);
    }
    sync();
  };
  // With flags, K is assembled by owned rows: warps 0-3 compute the rows of their CTA without the flags'
  // term under the flags' structural work on warps 4-7 (which takes longer than the body points), after a
  // barrier of warps 0-3 only (the published points are all this needs); the flags' term then comes from
  // the CTA's own columns of T J_d^-1 T^T (entry (r, c) from column r), and the rows are published before
  // the grid barrier that ends phase A, so phase B needs no barrier of its own.  Without flags, every
  // thread takes entries of the lower triangle (dense B0, both triangles written) or all entries (B0').
  const bool overlap_b = a.n_def > 0;

  bool converged = false;
  int it = 0, solves_total = 0, refreshes = 0;
  for (; it < a.max_iters; ++it) {
    // BIG with flags: the owned-row assembly below lists its near entries in the work area, over the cached owned
    // rows of X (every thread drops the copy, so all take the same reload branch at the next solve)
    if constexpr (BIG)
      if (overlap_b) xs_version = -1;
    // ---- A: body points, P, right-hand side.  Points are split over the CTAs (four threads per point, one
    // per hat vertex; FP64 throughput per SM is low on sm_103), published, then every CTA takes all of them.
    for (int bi = tid; bi < a.n_bodies; bi += nthr)
      if (a.bodies[bi].type == FSI_BODY_TORSIONAL) {
        if (kb_s) {  // moving hinge: rest direction of this step and g at the iterate
          double* k = kb_s + bi * KB_N;
          sincos(k[KB_T0] + b_th[bi], &b_sn[bi], &b_cs[bi]);
          double st, ct;
          sincos(b_th[bi], &st, &ct);
          k[KB_G] = k[KB_GX] * (-b_sn[bi]) + k[KB_GI] + k[KB_GC] * ct + k[KB_GS] * st;  // cos(alpha1 + theta) = -sin
        } else {
          sincos(a.bodies[bi].theta0 + b_th[bi], &b_sn[bi], &b_cs[bi]);
        }
      }
    __syncthreads();
    if constexpr (BIG) {
      for (int k = tid; k < nf; k += nthr) {
        const int p = k % nb, bb = pb_s[p];
        tors_s[k] = bt_s[bb] == FSI_BODY_TORSIONAL ? (double)(p - boff_s[bb]) * a.ds * (k < nb ? -b_sn[bb] : b_cs[bb])
                                                   : 0.0;
        torsf_s[k] = (float)tors_s[k];
      }
      __syncthreads();
    }
    {
      const int per = (nb + (int)gridDim.x - 1) / (int)gridDim.x;
      const int p0 = (int)blockIdx.x * per;
      // side timers of CTA 0 (slots 14: warps 0-3 on the points, 15: warps 4-7 on the flags)
      const bool side_clock = blockIdx.x == 0 && (tid == 0 || tid == 128) && a.phase_ns;
      const unsigned long long ta0 = side_clock ? PhaseClock::now() : 0ull;
      // warps 0-3 take the points (every lane of them joins the shuffles); warps 4-7 the flags
      for (int t0 = 0; wid < 4 && t0 < 4 * per; t0 += 128) {
        const int t = t0 + tid;
        const int p = p0 + (t >> 2), q = t & 3;
        const bool act = t < 4 * per && p < nb;
        double ubx = 0.0, uby = 0.0, svx = 0.0, svy = 0.0, ucx = 0.0, ucy = 0.0, coef = 0.0;
        if (act) {
          const int bi = a.point_body[p];
          const BodyDev b = a.bodies[bi];
          double x, y;
          if (b.type == FSI_BODY_TORSIONAL) {
            const double th_k = b_th[bi], ph_k = b_ph[bi];
            const int j = p - b.off;
            const double sn = b_sn[bi], cs = b_cs[bi];
            const double* k = kb_s ? kb_s + bi * KB_N : nullptr;
            x = (k ? k[KB_X] : b.hx) + (double)j * a.ds * cs;
            y = (k ? k[KB_Y] : b.hy) + (double)j * a.ds * sn;
            svx = (double)j * a.ds * (-sn);
            svy = (double)j * a.ds * cs;
            ucx = svx * ph_k;
            ucy = svy * ph_k;
            double rphik = b_rphi[bi] - b_jac[bi] * th_k;
            if (k) {  // moving hinge: its velocity and alpha1' q R, and g at the iterate
              ucx += k[KB_VX] + k[KB_AD] * svx;
              ucy += k[KB_VY] + k[KB_AD] * svy;
              rphik += k[KB_G];
            }
            const double rthk = b_rth[bi] - a.two_dt * th_k + ph_k;
            coef = rthk - a.two_dt * rphik * b_ijac[bi];
          } else if (b.type == FSI_BODY_DEFORMABLE) {  // node j of the flag at chi^(k); node 0 is the clamp
            const int j = p - b.off;
            x = j == 0 ? b.hx : chi_s[3 * (b.el_off + j - 1)];
            y = j == 0 ? b.hy : chi_s[3 * (b.el_off + j - 1) + 1];
          } else if (b.type == FSI_BODY_DRIVEN) {  // prescribed heave and pitch (Sec. 5.1)
            const double* k = kb_s + bi * KB_N;
            const double sj = b.s_lo + (double)(p - b.off) * a.ds;
            x = k[KB_X] + sj * k[KB_SA];
            y = k[KB_Y] - sj * k[KB_CA];
            ucx = k[KB_VX] + sj * k[KB_AD] * k[KB_CA];
            ucy = sj * k[KB_AD] * k[KB_SA];
          } else {
            x = a.rpts[2 * p];
            y = a.rpts[2 * p + 1];
            ucx = a.rur[2 * p];
            ucy = a.rur[2 * p + 1];
          }
          const int ap = a.app_idx ? a.app_idx[p] : -1;
          if (ap >= 0) {  // appended point (Sec. 3.1.1): its own unknown, weight one; E (C s* + q_inf) at it
            a.pidx[4 * p + q] = a.n_box + ap;
            a.pw[4 * p + q] = q == 0 ? 1.0 : 0.0;
            if (q == 0) {
              a.pcij[2 * p] = 0;
              a.pcij[2 * p + 1] = 0;
            }
            const FaceWindow W = a.app_win[ap];  // lane q takes row q of both 4 x 4 face windows
            for (int d = 0; d < 4; ++d) {
              const long Iu = W.iu + d, Ju = W.ju + q, Iv = W.iv + d, Jv = W.jv + q;
              const double u = (load_s(a, (Ju + 1) * a.ps + Iu) - load_s(a, Ju * a.ps + Iu)) / a.h + a.U;
              const double v = -(load_s(a, Jv * a.ps + Iv + 1) - load_s(a, Jv * a.ps + Iv)) / a.h + a.V;
              ubx += (W.w[d] * W.w[4 + q]) * u;
              uby += (W.w[8 + d] * W.w[12 + q]) * v;
            }
          }
          // the box holding the point: the only box, or the first box of a union that holds it; (ox, oy) its
          // corner in the bounding box, (bni, bnj) its vertex counts
          int ox = 0, oy = 0, bni = a.ni, bnj = a.nj;
          if (a.n_sdb > 1 && ap < 0) {
            int k = 0;
            for (int b = a.n_sdb - 1; b >= 0; --b) {
              const double gx = (x - (a.x0 + a.sdb[b][0] * a.h)) / a.h, gy = (y - (a.y0 + a.sdb[b][2] * a.h)) / a.h;
              if (gx >= 0.0 && gy >= 0.0 && gx <= (double)(a.sdb[b][1] - a.sdb[b][0]) &&
                  gy <= (double)(a.sdb[b][3] - a.sdb[b][2]))
                k = b;
            }
            ox = a.sdb[k][0] - a.i_lo;
            oy = a.sdb[k][2] - a.j_lo;
            bni = a.sdb[k][1] - a.sdb[k][0] + 1;
            bnj = a.sdb[k][3] - a.sdb[k][2] + 1;
          }
          const double xl = a.x0 + (a.i_lo + ox) * a.h, yl = a.y0 + (a.j_lo + oy) * a.h;
          const double fx = (x - xl) / a.h, fy = (y - yl) / a.h;
          int ci = (int)floor(fx), cj = (int)floor(fy);
          if (ap >= 0) {
          } else if (!(fx >= 0.0 && fy >= 0.0 && fx <= (double)(bni - 1) && fy <= (double)(bnj - 1))) {
            if (q == 0) dev_set_status(a.status, FSI_ERR_BODY_OUTSIDE_SUBDOMAIN);
            ci = 0;
            cj = 0;
          }
          ci = min(max(ci, 0), bni - 2);
          cj = min(max(cj, 0), bnj - 2);
          if (ap < 0) {
            const double rx = fx - ci, ry = fy - cj;
            const int aa = q & 1, bb = q >> 1;
            const double wq = (aa ? rx : 1.0 - rx) * (bb ? ry : 1.0 - ry);
            const int vi = ox + ci + aa, vj = oy + cj + bb;  // hat vertex in the bounding box
            a.pidx[4 * p + q] = a.sd_map ? a.sd_map[vj * a.ni + vi] : vj * a.ni + vi;
            a.pw[4 * p + q] = wq;
            if (q == 0) {
              a.pcij[2 * p] = ox + ci;
              a.pcij[2 * p + 1] = oy + cj;
            }
            double u, v;
            e0cs(a, a.i_lo + vi, a.j_lo + vj, &u, &v);
            ubx = wq * u;
            uby = wq * v;
          }
        }
        // sum over the four hat vertices in the fixed order ((q0 + q1) + (q2 + q3))
        ubx += __shfl_xor_sync(FULL, ubx, 1);
        uby += __shfl_xor_sync(FULL, uby, 1);
        ubx += __shfl_xor_sync(FULL, ubx, 2);
        uby += __shfl_xor_sync(FULL, uby, 2);
        if (act && q == 0) {
          a.rhs[2 * nf + p] = ubx - ucx + svx * coef;
          a.rhs[2 * nf + nb + p] = uby - ucy + svy * coef;
        }
      }
      unsigned long long tb = side_clock ? PhaseClock::now() : 0ull;
      if (side_clock && tid == 0) sh_phase[14] += tb - ta0;
      auto side_sub = [&](int slot) {  // consecutive sub-steps of phase A on thread 0 of CTA 0
        if (side_clock && tid == 0) {
          const unsigned long long t = PhaseClock::now();
          sh_phase[slot] += t - tb;
          tb = t;
        }
      };
      if (overlap_b && wid < 4) {
        lower_grid_barrier(&a.ctrl[15], (it + 1) * (int)gridDim.x + a.lb_missing, a.status, a.lb_spins);
        side_sub(16);
        for (int e0 = tid; e0 < 4 * nb; e0 += 128 * 8) {  // eight entries' loads in flight per thread
          int iv[8];
          double wv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = e0 + 128 * u;
            iv[u] = e < 4 * nb ? __ldcg(&a.pidx[e]) : 0;
            wv[u] = e < 4 * nb ? __ldcg(&a.pw[e]) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int e = e0 + 128 * u;
            if (e < 4 * nb) {
              pidx_s[e] = iv[u];
              pw_s[e] = wv[u];
            }
          }
        }
        for (int e0 = tid; e0 < 2 * nb; e0 += 128 * 8) {
          int cv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) cv[u] = e0 + 128 * u < 2 * nb ? __ldcg(&a.pcij[e0 + 128 * u]) : 0;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (e0 + 128 * u < 2 * nb) pcij_s[e0 + 128 * u] = cv[u];
        }
        named_sync_lower();
        body_boxes(tid, 128, []() { named_sync_lower(); });
        side_sub(17);
        if constexpr (BIG) {
          // Owned rows stay in global memory, body block by body block: the blocks of bodies that do not couple
          // (Omega_0 hat cells farther apart than the B0' window) are zero and cost one store per entry.  S, the
          // float copy, is written here except where a flag's structural term is still to come.  Two passes:
          // (1) every entry without its window term -- zero, or the torsional rank-one term (one FP64 multiply-add
          // with the row's factor hoisted; its float copy a float product, since FP64 instructions and
          // double-to-float conversions run at a small fraction of the FP32 rate on this GPU) -- while the near
          // entries (hat cells within the window: a band of ~2 x 29 columns around a row's own point) are listed
          // in shared memory; (2) the listed entries dealt evenly over the threads, two per thread at a time with
          // the loads of both windows issued before either is summed.  (Computed where they fall in the rows, a
          // warp meets near entries in one or two of its column steps of every row, and each such step waits a
          // full memory latency for its few lanes.)  The list lives in the work area that caches the owned rows
          // of X between its changes, so that copy is reloaded at the next solve; entries beyond its capacity
          // are computed in pass 1.
          const double kscale = a.ds / (a.h * a.h);
          __shared__ int n_near;
          int* nlist = reinterpret_cast<int*>(tile);
          const int ncap = nf < 65536 ? (int)fsi_big_work_floats(a.nbody_max) : 0;  // (row, column) in one int
          if (tid == 0) n_near = 0;
          named_sync_lower();
          for (int c = 0; c < nr; ++c) {
            const int r = r0 + c, ca = r >= nb ? 1 : 0, pa = r - ca * nb, ba = pb_s[pa];
            const int cia = pcij_s[2 * pa], cja = pcij_s[2 * pa + 1];
            const double ka = bt_s[ba] == FSI_BODY_TORSIONAL ? b_kc[ba] * tors_s[r] : 0.0;
            const float kaf = (float)ka;
            double* kr = a.K + (long)r * nf;
            float* sr = a.S + (long)r * lx;
            for (int bb = 0; bb < a.n_bodies; ++bb) {
              const int n = bn_s[bb], off = boff_s[bb];
              const bool cp = couples(ba, bb), later = cp && ba == bb && bt_s[bb] == FSI_BODY_DEFORMABLE;
              const bool rank1 = cp && ba == bb && bt_s[bb] == FSI_BODY_TORSIONAL;
              // a block of bodies that do not couple is read by nothing in the solve (residual rows, block
              // products and rebuild take the coupled and diagonal blocks): its zeros are written in the first
              // iteration of a launch only, for fsi_get_small_system
              if (!cp && it > 0) continue;
              for (int t = tid; t < 2 * n; t += 128) {
                const int cb = t >= n ? 1 : 0, pb = off + t - cb * n, cidx = cb * nb + pb;
                bool nz = false;
                if (cp) {  // cp is the same in every thread
                  const int dj0 = cja - pcij_s[2 * pb + 1], di0 = cia - pcij_s[2 * pb];
                  nz = dense || window_near(dj0, di0);
                  // list slots taken warp by warp: one shared-memory atomic per warp step (per-lane atomics on
                  // the one counter serialise)
                  const unsigned act = __activemask(), m = __ballot_sync(act, nz);
                  if (m) {
                    const int lead = __ffs(act) - 1;
                    int base = 0;
                    if (lane == lead) base = atomicAdd(&n_near, __popc(m));
                    base = __shfl_sync(act, base, lead);
                    const int q = base + __popc(m & ((1u << lane) - 1u));
                    if (nz && q < ncap) {
                      nlist[q] = (c << 16) | cidx;
                      continue;
                    }
                  }
                }
                double kv = 0.0;
                float sv = 0.0f;
                if (nz) {  // beyond the list's capacity
                  const double acc = dense ? k_entry(r, cidx, false, true)
                                           : window_acc(pa, ca, pb, cb, cja - pcij_s[2 * pb + 1], cia - pcij_s[2 * pb]);
                  kv = acc != 0.0 ? kscale * acc : 0.0;
                }
                if (rank1) kv += ka * tors_s[cidx];
                if (nz) sv = (float)kv;
                else if (rank1) sv = kaf * torsf_s[cidx];
                kr[cidx] = kv;
                if (!later) sr[cidx] = sv;
              }
            }
          }
          named_sync_lower();
          const int nn = min(n_near, ncap);
          for (int q0 = tid; q0 < nn; q0 += 256) {
            int cq[2], idq[2], dj[2], di[2];
            bool on[2];
            double v[2][16];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int q = q0 + 128 * u;
              on[u] = q < nn;
              const int e = on[u] ? nlist[q] : 0;
              cq[u] = e >> 16;
              idq[u] = e & 0xffff;
              const int r = r0 + cq[u], ca = r >= nb ? 1 : 0, pa = r - ca * nb;
              const int cb = idq[u] >= nb ? 1 : 0, pb = idq[u] - cb * nb;
              dj[u] = pcij_s[2 * pa + 1] - pcij_s[2 * pb + 1];
              di[u] = pcij_s[2 * pa] - pcij_s[2 * pb];
              window_load(ca, pb, cb, dj[u], di[u], on[u] && !dense, v[u]);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              if (!on[u]) continue;
              const int c = cq[u], r = r0 + c, ca = r >= nb ? 1 : 0, pa = r - ca * nb, ba = pb_s[pa];
              const int cidx = idq[u], cb = cidx >= nb ? 1 : 0, pb = cidx - cb * nb, bb = pb_s[pb];
              const double acc = dense ? k_entry(r, cidx, false, true) : window_sum(pa, pb, dj[u], di[u], v[u]);
              double kv = acc != 0.0 ? kscale * acc : 0.0;
              if (ba == bb && bt_s[bb] == FSI_BODY_TORSIONAL) kv += (b_kc[ba] * tors_s[r]) * tors_s[cidx];
              a.K[(long)r * nf + cidx] = kv;
              if (!(ba == bb && bt_s[bb] == FSI_BODY_DEFORMABLE)) a.S[(long)r * lx + cidx] = (float)kv;
            }
          }
        } else {
          for (int e = tid; e < nr * nf; e += 128) {
            const int r = r0 + e / nf, cidx = e % nf;
            Krow[e] = couples(pb_s[r % nb], pb_s[cidx % nb]) ? k_entry(r, cidx, false) : 0.0;
          }
        }
        side_sub(18);
      }
      if (wid >= 4 && a.n_def > 0) {
        // ---- A': every flag linearised at chi^(k) (warps 4-7): element forces (FP64) and tangents (FP32),
        // r^zeta(k), J_d blocks, the factorization, y = J_d^-1 (r^zeta(k) + ds T^T f_prev) and the structural
        // columns of the owned rows.
        const int st = tid - 128;
        for (int bi = 0; bi < a.n_bodies; ++bi) {
          const BodyDev b = a.bodies[bi];
          if (b.type != FSI_BODY_DEFORMABLE) continue;
          const int N = b.n - 1, e0 = b.el_off, d0 = 3 * e0, ld = 3 * N;
          float* ey = ey_s + 12 * e0;  // element tangents [N][aa 6 | bb 6], later [Em 9N | y 3N]
          const beam::Flag F{N,
                             b.hx,
                             b.hy,
                             b.mu,
                             a.ds,
                             beam::ElemParams{a.ds, b.ea / a.ds, 2.0 * b.ei / a.ds},
                             a.four_dt2,
                             2.0 * a.two_dt,
                             chi_s + d0,
                             ref_s + 3 * e0,
                             cn_s + d0,
                             fab_s + 6 * e0,
                             ey,
                             mi_s + 6 * e0,
                             bm_s + 9 * e0,
                             rz_s + d0,
                             ys_s,
                             f_s + b.off + 1,
                             nb};
          beam::flag_elements(F, st, 128);
          named_sync_upper();
          int nrhs = 1, rdof[MR], rrow[MR];  // owned structural columns of this flag
#pragma unroll
          for (int c = 0; c < MR; ++c)
            if (g_body[c] == bi) {
              rdof[nrhs - 1] = g_dof[c];
              rrow[nrhs - 1] = r0 + c;
              ++nrhs;
            }
          beam::flag_assemble(F, st, 128);
          for (int q = st; q < ld; q += 128)  // unit right-hand sides of the owned columns
            for (int j = 1; j < nrhs; ++j) ys_s[j * ld + q] = q == rdof[j - 1] ? 1.f : 0.f;
          named_sync_upper();
          {
            const beam::Bcr B = beam::flag_bcr(F);
            beam::bcr_factor(B, st, 128, []() { named_sync_upper(); });
            beam::bcr_solve(B, ys_s, ld, nrhs, st, 128, []() { named_sync_upper(); });
          }
          float* ysol = ey + 9 * N;
          for (int q = st; q < ld; q += 128) ysol[q] = ys_s[q];
          for (int j = 1; j < nrhs; ++j) {
            double* col = a.G + (long)rrow[j - 1] * nf;
            for (int i = st; i < N; i += 128) {
              col[b.off + 1 + i] = (double)ys_s[j * ld + 3 * i];
              col[nb + b.off + 1 + i] = (double)ys_s[j * ld + 3 * i + 1];
            }
          }
          named_sync_upper();
        }
        if (side_clock) sh_phase[15] += PhaseClock::now() - ta0;
      }
    }
    const bool pclk = blockIdx.x == 0 && tid == 0 && a.phase_ns;
    unsigned long long tc = pclk ? PhaseClock::now() : 0ull;
    auto a_sub = [&](int slot) {
      if (pclk) {
        const unsigned long long t = PhaseClock::now();
        sh_phase[slot] += t - tc;
        tc = t;
      }
    };
    if (overlap_b) {  // owned rows: the flags' term from this CTA's columns of T J_d^-1 T^T, then publish
      __syncthreads();
      a_sub(19);
      if constexpr (BIG) {  // only a flag's own block receives the term
        // four owned rows at a time, every K and G entry of the four loaded before any is updated (one memory
        // latency per four rows instead of one per row)
        const double gsc = a.ds * a.two_dt;
        bool any_flag = false;  // an owned row of a flag (the same in every thread)
        for (int c = 0; c < nr; ++c) any_flag = any_flag || bt_s[pb_s[(r0 + c) % nb]] == FSI_BODY_DEFORMABLE;
        for (int c0 = 0; any_flag && c0 < nr; c0 += 4)
          for (int tb = 0; tb < 2 * a.nbody_max; tb += 2 * nthr) {
            double kv[4][2], gv[4][2];
            long ik[4][2], is[4][2];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int c = c0 + u, r = r0 + c, ba = c < nr ? pb_s[r % nb] : 0;
              const int n = c < nr && bt_s[ba] == FSI_BODY_DEFORMABLE ? bn_s[ba] : 0, off = boff_s[ba];
#pragma unroll
              for (int v = 0; v < 2; ++v) {
                const int t = tb + tid + v * nthr;
                const int cidx = t < n ? off + t : nb + off + t - n;
                ik[u][v] = t < 2 * n ? (long)r * nf + cidx : -1;
                is[u][v] = t < 2 * n ? (long)r * lx + cidx : -1;
                kv[u][v] = t < 2 * n ? a.K[ik[u][v]] : 0.0;
                gv[u][v] = t < 2 * n ? __ldcg(&a.G[ik[u][v]]) : 0.0;
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 2; ++v) {
                if (ik[u][v] < 0) continue;
                const double k = kv[u][v] + gsc * gv[u][v];
                a.K[ik[u][v]] = k;
                a.S[is[u][v]] = (float)k;
              }
          }
      } else {
        for (int e = tid; e < nr * nf; e += nthr) {
          const int r = r0 + e / nf, cidx = e % nf;
          double kv = Krow[e];
          const int ba = a.point_body[r % nb];
          if (ba == a.point_body[cidx % nb] && a.bodies[ba].type == FSI_BODY_DEFORMABLE)
            kv += a.ds * a.two_dt * __ldcg(&a.G[(long)r * nf + cidx]);
          Krow[e] = kv;
          a.K[(long)r * nf + cidx] = kv;
          a.S[(long)r * lx + cidx] = (float)kv;
        }
      }
      a_sub(20);
    }
    grid.sync();
    a_sub(21);
    if (!overlap_b) {
      for (int e = tid; e < 4 * nb; e += nthr) {
        pidx_s[e] = __ldcg(&a.pidx[e]);
        pw_s[e] = __ldcg(&a.pw[e]);
      }
      for (int e = tid; e < 2 * nb; e += nthr) pcij_s[e] = __ldcg(&a.pcij[e]);
      __syncthreads();
      body_boxes(tid, nthr, []() { __syncthreads(); });
    }
    for (int e = tid; e < nf; e += nthr) rhs_s[e] = __ldcg(&a.rhs[2 * nf + e]);
    __syncthreads();
    if (a.n_def > 0) {  // flags: rhs -= T ((2/dt)(chi^(k) + y) - r^chi_n)
      for (int bi = 0; bi < a.n_bodies; ++bi) {
        const BodyDev b = a.bodies[bi];
        if (b.type != FSI_BODY_DEFORMABLE) continue;
        const int N = b.n - 1, d0 = 3 * b.el_off;
        const float* ysol = ey_s + 12 * b.el_off + 9 * N;
        for (int q = tid; q < 2 * N; q += nthr) {
          const int i = q >> 1, c = q & 1, g = d0 + 3 * i + c;
          rhs_s[c * nb + b.off + 1 + i] -= a.two_dt * (chi_s[g] + (double)ysol[3 * i + c]) - rchi_s[g];
        }
      }
      __syncthreads();
    }
    a_sub(22);
    clk.mark(0);
    // ---- B: K = (ds/h^2) P B0 P^T + (2 ds/dt) S^T J^{-1} S (with flags already assembled by owned rows)
    if (!overlap_b && BIG) {  // owned rows, body block by body block (see the flags' variant above)
      for (int c = 0; c < nr; ++c) {
        const int r = r0 + c, ba = pb_s[r % nb];
        for (int bb = 0; bb < a.n_bodies; ++bb) {
          const int n = bn_s[bb], off = boff_s[bb];
          const bool cp = couples(ba, bb);
          if (!cp && it > 0) continue;  // zeros written once per launch (see the flags' variant)
          for (int t = tid; t < 2 * n; t += nthr) {
            const int cidx = t < n ? off + t : nb + off + t - n;
            const double kv = cp ? k_entry(r, cidx, true) : 0.0;
            a.K[(long)r * nf + cidx] = kv;
            a.S[(long)r * lx + cidx] = (float)kv;
          }
        }
      }
      grid.sync();
    } else if (!overlap_b) {
      for (long e = gtid; e < (long)nf * nf; e += gsize) {
        const int r = (int)(e / nf), cidx = (int)(e % nf);
        if (dense && cidx > r) continue;
        const double kv = couples(pb_s[r % nb], pb_s[cidx % nb]) ? k_entry(r, cidx, true) : 0.0;
        a.K[(long)r * nf + cidx] = kv;
        a.S[(long)r * lx + cidx] = (float)kv;
        if (dense) {
          a.K[(long)cidx * nf + r] = kv;
          a.S[(long)cidx * lx + r] = (float)kv;
        }
      }
      grid.sync();
      if constexpr (!BIG)
        for (int e = tid; e < nr * nf; e += nthr) Krow[e] = __ldcg(&a.K[(long)r0 * nf + e]);  // owned rows of K
    }
    // Flags.  The structural right-hand side was formed from J_d^-1 (r^zeta(k) + ds T^T f_prev) instead of
    // J_d^-1 r^zeta(k); the two differ by (2 ds/dt) T J_d^-1 T^T f_prev, which the owned residual rows add
    // back here with the same entries of T J_d^-1 T^T that K holds.  Both FP32 structural solves then act
    // on quantities that vanish at the fixed point, whose float errors therefore vanish with them.
    __shared__ double gfp_s[MR];
    if (a.n_def > 0) {
      for (int c = wid; c < MR; c += nw) {
        double acc = 0.0;
        if (c < nr) {
          const int r = r0 + c;
          const BodyDev b = a.bodies[a.point_body[r % nb]];
          if (b.type == FSI_BODY_DEFORMABLE)
            for (int q = lane; q < 2 * b.n; q += 32) {
              const int m = q < b.n ? b.off + q : nb + b.off + q - b.n;
              // the entry K holds: column r (owned-row assembly) or column min(r, m) (lower triangle)
              const long gi = overlap_b || r < m ? (long)r * nf + m : (long)m * nf + r;
              acc += __ldcg(&a.G[gi]) * f_s[m];
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) gfp_s[c] = a.ds * a.two_dt * acc;
      }
    } else if (tid < MR) {
      gfp_s[tid] = 0.0;
    }
    __syncthreads();
    clk.mark(1);
    // ---- C: refresh the float inverse (Newton-Schulz from the previous one, or a rebuild), then refine
    // Newton-Schulz refresh of the float inverse for the current K: X <- 2X - (X K) X, kNsSteps times
    // BIG: one Newton-Schulz step on every block, T = X K then X <- 2X - T X, by owned rows
    auto big_ns_step = [&]() {
      float* Xc = cur ? a.Xb : a.Xa;
      float* Xn = cur ? a.Xa : a.Xb;
      blk_gemm(a, Xc, a.S, Xc, 0.0f, 1.0f, a.T, lx, tile);
      grid.sync();
      clk.sub(8);
      blk_gemm(a, a.T, Xc, Xc, 2.0f, -1.0f, Xn, lx, tile);
      grid.sync();
      clk.sub(9);
      cur ^= 1;
      ++x_version;
    };
    auto ns_refresh = [&]() {
      if constexpr (BIG) {  // one step: the error I - K X is squared, and a step costs four block GEMMs
        big_ns_step();
      } else {
        for (int ns = 0; ns < kNsSteps; ++ns) {  // X <- 2X - (X K) X: the error I - K X is squared
          float* Xn = cur ? a.Xa : a.Xb;
          // (a) owned columns of T = X K: T[i][r0 + c] = sum_m X[i][m] K[m][r0 + c]
          for (int m = tid; m < lx; m += nthr) {  // entries m >= nf stay zero
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            const float* kr = a.S + (long)m * lx + r0;
            if (m < nf && nr > 0) v.x = __ldcg(kr);
            if (m < nf && nr > 1) v.y = __ldcg(kr + 1);
            if (m < nf && nr > 2) v.z = __ldcg(kr + 2);
            if (m < nf && nr > 3) v.w = __ldcg(kr + 3);
            work4[m] = v;
          }
          __syncthreads();
          if (nr > 0) {
            for (int i = tid; i < nf; i += nthr) {  // thread per row i, 128-bit loads (conflict-free stride)
              float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
              const float4* xr = reinterpret_cast<const float4*>(Xs + (long)i * lx);
              for (int m4 = 0; m4 < lx / 4; ++m4) {
                const float4 xv = xr[m4];
                const float4 k0 = work4[4 * m4], k1 = work4[4 * m4 + 1], k2 = work4[4 * m4 + 2], k3 = work4[4 * m4 + 3];
                acc.x += xv.x * k0.x + xv.y * k1.x + xv.z * k2.x + xv.w * k3.x;
                acc.y += xv.x * k0.y + xv.y * k1.y + xv.z * k2.y + xv.w * k3.y;
                acc.z += xv.x * k0.z + xv.y * k1.z + xv.z * k2.z + xv.w * k3.z;
                acc.w += xv.x * k0.w + xv.y * k1.w + xv.z * k2.w + xv.w * k3.w;
              }
              float* tr = a.T + (long)i * lx + r0;
              tr[0] = acc.x;
              if (nr > 1) tr[1] = acc.y;
              if (nr > 2) tr[2] = acc.z;
              if (nr > 3) tr[3] = acc.w;
            }
          }
          grid.sync();
          clk.sub(8);
          // (b) owned rows of the new X: Xn[r0 + c][j] = 2 X[r0 + c][j] - sum_m T[r0 + c][m] X[m][j]
          for (int m = tid; m < nf; m += nthr) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (nr > 0) v.x = __ldcg(&a.T[(long)r0 * lx + m]);
            if (nr > 1) v.y = __ldcg(&a.T[(long)(r0 + 1) * lx + m]);
            if (nr > 2) v.z = __ldcg(&a.T[(long)(r0 + 2) * lx + m]);
            if (nr > 3) v.w = __ldcg(&a.T[(long)(r0 + 3) * lx + m]);
            work4[m] = v;
          }
          __syncthreads();
          if (nr > 0) {
            for (int j = tid; j < nf; j += nthr) {
              float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  #pragma unroll 4
              for (int m = 0; m < nf; ++m) {
                const float xv = Xs[(long)m * lx + j];
                const float4 tv = work4[m];
                acc.x += tv.x * xv;
                acc.y += tv.y * xv;
                acc.z += tv.z * xv;
                acc.w += tv.w * xv;
              }
              Xn[(long)r0 * lx + j] = 2.0f * Xs[(long)r0 * lx + j] - acc.x;
              if (nr > 1) Xn[(long)(r0 + 1) * lx + j] = 2.0f * Xs[(long)(r0 + 1) * lx + j] - acc.y;
              if (nr > 2) Xn[(long)(r0 + 2) * lx + j] = 2.0f * Xs[(long)(r0 + 2) * lx + j] - acc.z;
              if (nr > 3) Xn[(long)(r0 + 3) * lx + j] = 2.0f * Xs[(long)(r0 + 3) * lx + j] - acc.w;
            }
          }
          grid.sync();
          clk.sub(9);
          load_x(Xs, Xn, nf, lx, &xbar, &xphase, a.status);  // (c) every CTA takes the whole new X
          __syncthreads();
          clk.sub(10);
          cur ^= 1;
        }
      }
      clk.mark(2);
    };
    for (int attempt = 0; attempt < 2; ++attempt) {
      bool fresh = false;  // X was refreshed or rebuilt for this K
      int n_refresh = 0;   // Newton-Schulz refreshes in this attempt (the distributed variant allows several)
      if (BIG && !kinv_valid) {
        // X0 = alpha I on every block with alpha = 1 / (largest absolute row sum of the block of K), so that the
        // eigenvalues of alpha K lie in the unit disc about 1, then Newton-Schulz steps to convergence
        for (int c = wid; c < nr; c += nw) {
          const int i = r0 + c;
          const RowBlock b = row_block(a, i);
          double acc = 0.0;
          for (int t = lane; t < 2 * b.n; t += 32) acc += fabs(__ldcg(&a.K[(long)i * nf + blk_col(b, nb, t)]));
          acc = warp_sum(acc);
          if (lane == 0) a.rsum[i] = acc;
        }
        grid.sync();
        float* Xc = cur ? a.Xb : a.Xa;
        for_groups([&](int g0, int ng, RowBlock b) {
          double mx = 0.0;
          for (int t = tid; t < 2 * b.n; t += nthr) mx = fmax(mx, __ldcg(&a.rsum[blk_col(b, nb, t)]));
          mx = block_max(mx, red);
          const float alpha = (float)(1.0 / mx);
          for (int e = tid; e < ng * 2 * b.n; e += nthr) {
            const int g = e / (2 * b.n), t = e - g * 2 * b.n, col = blk_col(b, nb, t);
            Xc[(long)(g0 + g) * lx + col] = col == g0 + g ? alpha : 0.0f;
          }
          __syncthreads();
        });
        grid.sync();
        for (int k = 0; k < kNsRebuild; ++k) big_ns_step();
        kinv_valid = 1;
        fresh = true;
        if (blockIdx.x == 0 && tid == 0) a.ctrl[6] += 1;  // rebuild count
        clk.mark(3);
      }
      if (!BIG && !kinv_valid) {
        float* Lf = Xs;  // CTA 0 factors in the space of X, which is being rebuilt
        if (blockIdx.x == 0) {
          for (int i = tid >> 5; i < nf; i += nthr >> 5)
            for (int k = lane; k <= i; k += 32)  // the symmetric part of K (K itself for the dense B0
                                                 // without flags; with flags K is symmetric only to FP32
                                                 // rounding of its structural columns)
              Lf[(long)i * ld + k] =
                  (float)(0.5 * (__ldcg(&a.K[(long)i * nf + k]) + __ldcg(&a.K[(long)k * nf + i])));
          __syncthreads();
          chol_blocked(Lf, nf, ld, &sh_bad);
          tri_inverse(Lf, nf, ld, a.T);
        }
        grid.sync();
        float* Xc = cur ? a.Xb : a.Xa;
        for (long i = wg; i < nf; i += nwg) {  // X = W^T W, warp per row i, lanes over k <= i
          for (int k0 = 0; k0 <= i; k0 += 32) {
            const int k = k0 + lane;
            float acc = 0.0f;
            if (k <= i)
              for (int m = (int)i; m < nf; ++m) acc += __ldcg(&a.T[(long)m * nf + i]) * __ldcg(&a.T[(long)m * nf + k]);
            if (k <= i) {
              Xc[i * lx + k] = acc;
              Xc[(long)k * lx + i] = acc;
            }
          }
        }
        grid.sync();
        load_x(Xs, Xc, nf, lx, &xbar, &xphase, a.status);
        __syncthreads();
        kinv_valid = 1;
        fresh = true;
        if (blockIdx.x == 0 && tid == 0) a.ctrl[6] += 1;  // rebuild count
        clk.mark(3);
      }
      bool done = false, bad = false;
      int s = 0;
      double gd_prev = 0.0, worst_ratio = 0.0;
      const bool warm = a.n_def > 0;  // start from f_prev: one residual (and barrier) before the first solve
      if (warm) {
        if (attempt > 0) {
          for (int k = tid; k < nf; k += nthr) f_s[k] = 0.0;
          __syncthreads();
        }
        for (int c = wid; c < nr; c += nw) {
          double acc = 0.0;
          if constexpr (BIG) {
            acc = coupled_dot(r0 + c);
          } else {
            const double* kr = Krow + (long)c * nf;
            for (int k = lane; k < nf; k += 32) acc += kr[k] * f_s[k];
          }
          acc = warp_sum(acc);
          if (lane == 0) {
            const double rv = rhs_s[r0 + c] + gfp_s[c] - acc;
            res1[r0 + c] = rv;
            if constexpr (BIG) a.resf[nf + r0 + c] = (float)rv;
          }
        }
        grid.sync();
        if constexpr (BIG)
          gather_f(rf, a.resf + nf, nf);
        else
          for (int k = tid; k < nf; k += nthr) r_s[k] = __ldcg(&res1[k]);
        __syncthreads();
      }
      for (; s < kMaxSolves; ++s) {
        if (!BIG || (s == 0 && !warm)) {  // the distributed variant gathered the float residual already
          const double* r = (s == 0 && !warm) ? rhs_s : r_s;
          for (int k = tid; k < nf; k += nthr) rf[k] = (float)r[k];
        }
        __syncthreads();
        unsigned dbits = 0u, xbits = 0u;  // max |d|, max |f| as float bit patterns
        unsigned long long dbits64 = 0ull, xbits64 = 0ull;  // the same as double bit patterns (BIG)
        if constexpr (BIG) {  // owned rows of d = X r (block columns), shared through global memory
          const float* Xc = cur ? a.Xb : a.Xa;
          // X changes only at a Newton-Schulz step or a rebuild, once or twice a time step, while a dozen
          // solves apply it: each CTA keeps its owned rows' blocks of X in shared memory (the block products'
          // tile area) from one change to the next.  (Read from global memory in every solve, the loads of
          // this register-heavy kernel stay nearly serialised: 6.3 us per solve against 0.8 us for the same
          // loop in a light kernel.)
          const int w2 = 2 * a.nbody_max;
          if (xs_version != x_version) {
            for (int e = tid; e < nr * w2; e += nthr) {
              const int c = e / w2, t = e - c * w2, i = r0 + c, bi = pb_s[i % nb];
              const RowBlock b{boff_s[bi], bn_s[bi]};
              if (t < 2 * b.n) tile[e] = __ldcg(&Xc[(long)i * lx + blk_col(b, nb, t)]);
            }
            __syncthreads();
            xs_version = x_version;
          }
          for (int c = wid; c < nr; c += nw) {
            const int i = r0 + c, bi = pb_s[i % nb];
            const RowBlock b{boff_s[bi], bn_s[bi]};
            const float* xs = tile + c * w2;
            float acc = 0.0f;
            for (int t = lane; t < 2 * b.n; t += 32) acc += xs[t] * rf[blk_col(b, nb, t)];
            acc = warp_sum_f(acc);
            if (lane == 0) a.dvec[i] = (double)acc;
          }
          grid.sync();
          clk.sub(23);
          // the maxima on the bit patterns of |d| and |f| (integer operations: no conversions), a non-finite
          // f recorded as infinity
          constexpr unsigned long long kAbs = 0x7fffffffffffffffull, kInf = 0x7ff0000000000000ull;
          for (int i0 = tid; i0 < nf; i0 += nthr * 8) {  // the thread's loads issued together
            double dv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) dv[u] = i0 + u * nthr < nf ? __ldcg(&a.dvec[i0 + u * nthr]) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int i = i0 + u * nthr;
              if (i >= nf) break;
              const double di = dv[u];
              const double xi = (s == 0 && !warm ? 0.0 : f_s[i]) + di;
              f_s[i] = xi;
              const unsigned long long xb = (unsigned long long)__double_as_longlong(xi) & kAbs;
              const unsigned long long db = (unsigned long long)__double_as_longlong(di) & kAbs;
              dbits64 = max(dbits64, xb >= kInf ? kInf : db);
              xbits64 = max(xbits64, xb);
            }
          }
        }
        for (int i = BIG ? nf : tid; i < nf; i += nthr) {  // d = X r, f += d (every CTA, all rows; thread per row)
          const float4* xr = reinterpret_cast<const float4*>(Xs + (long)i * lx);
          const float4* r4 = reinterpret_cast<const float4*>(rf);
          float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;  // four chains, summed in a fixed order
          for (int k4 = 0; k4 < lx / 4; ++k4) {
            const float4 xv = xr[k4], rv = r4[k4];
            p0 += xv.x * rv.x;
            p1 += xv.y * rv.y;
            p2 += xv.z * rv.z;
            p3 += xv.w * rv.w;
          }
          const float acc = (p0 + p1) + (p2 + p3);
          const double xi = (s == 0 && !warm ? 0.0 : f_s[i]) + (double)acc;
          f_s[i] = xi;
          const float xf = (float)xi;
          dbits = max(dbits, isfinite(xf) ? __float_as_uint(fabsf(acc)) : 0x7f800000u);
          xbits = max(xbits, __float_as_uint(fabsf(xf)));
        }
        double gd, gx;
        if constexpr (BIG) {
          block_max2_bits64(dbits64, xbits64, red);
          gd = __longlong_as_double((long long)dbits64);
          gx = __longlong_as_double((long long)xbits64);
        } else {
          block_max2_bits(dbits, xbits, redu);
          gd = (double)__uint_as_float(dbits);
          gx = (double)__uint_as_float(xbits);
        }
        clk.sub(11);
        clk.mark(4);
        if (!isfinite(gd)) {  // a diverged inverse: rebuild and retry
          bad = true;
          break;
        }
        const double ratio = (s > 0 && gd_prev > 0.0) ? gd / gd_prev : 0.0;
        gd_prev = gd;
        if (gd <= kRefineTol * gx) {
          if (s > 0) worst_ratio = fmax(worst_ratio, ratio);
          done = true;
          break;
        }
        if (s == kMaxSolves - 1) break;
        // X is stale for this K: refresh it, keep f and r (the distributed variant tolerates a slower
        // contraction before paying for its block GEMMs, and refreshes again, up to kMaxRefreshB times, while
        // the contraction measured after a refresh stays above its trigger)
        if ((BIG ? n_refresh < kMaxRefreshB : !fresh) && s > 0 && ratio > (BIG ? 0.05 : kNsTrigger)) {
          ns_refresh();
          ++refreshes;
          ++n_refresh;
          fresh = true;
          gd_prev = 0.0;  // the next correction is the first one made with the new X: no ratio for it
        } else if (s > 0) {
          worst_ratio = fmax(worst_ratio, ratio);
        }
        for (int c = wid; c < nr; c += nw) {  // owned residual rows r = rhs - K f in double
          double acc = 0.0;
          if constexpr (BIG) {
            acc = coupled_dot(r0 + c);
          } else {
            const double* kr = Krow + (long)c * nf;
            for (int k = lane; k < nf; k += 32) acc += kr[k] * f_s[k];
          }
          acc = warp_sum(acc);
          if (lane == 0) {
            const double rv = rhs_s[r0 + c] + gfp_s[c] - acc;
            ((s & 1) ? res1 : res0)[r0 + c] = rv;
            if constexpr (BIG) a.resf[(s & 1) * nf + r0 + c] = (float)rv;
          }
        }
        grid.sync();
        clk.sub(12);
        if constexpr (BIG) {  // the float residual is all the next solve needs
          gather_f(rf, a.resf + (s & 1) * nf, nf);
        } else {
          const double* rg = (s & 1) ? res1 : res0;
          for (int k = tid; k < nf; k += nthr) r_s[k] = __ldcg(&rg[k]);
        }
        __syncthreads();
        clk.sub(13);
        clk.mark(5);
      }
      solves_total += s + 1;
      if (done) {
        // a slow contraction marks X for a rebuild at the next iteration; the distributed variant refreshes it
        // there instead (its rebuild starts from a scaled identity)
        if (!BIG && worst_ratio > kStaleRatio) kinv_valid = 0;
        break;
      }
      kinv_valid = 0;  // not converged with this inverse: rebuild it and solve again
      if (attempt == 1 && blockIdx.x == 0 && tid == 0)
        dev_set_status(a.status, bad ? FSI_ERR_NONFINITE : FSI_ERR_NOT_CONVERGED);
    }
    // ---- D: dtheta per torsional body (Eq. dtheta2), dchi per flag (Eq. dchi2), convergence on the largest
    // update (same in every CTA)
    double dmax = 0.0;
    bool finite = true;
    for (int bi = 0; bi < a.n_bodies; ++bi) {
      const BodyDev b = a.bodies[bi];
      if (b.type == FSI_BODY_DEFORMABLE) {  // dchi = J_d^-1 (r^zeta(k) + ds T^T f)
        const int N = b.n - 1, e0 = b.el_off, d0 = 3 * e0;
        for (int q = tid; q < 3 * N; q += nthr) {
          const int i = q / 3, k = q - 3 * i;
          double v = rz_s[d0 + q];
          if (k < 2) v += a.ds * f_s[k * nb + b.off + 1 + i];
          ys_s[q] = (float)v;
        }
        __syncthreads();
        beam::bcr_solve(beam::Bcr{mi_s + 6 * e0, bm_s + 9 * e0, ey_s + 12 * e0, N}, ys_s, 3 * N, 1, tid, nthr,
                        []() { __syncthreads(); });
        double dm = 0.0;
        for (int q = tid; q < 3 * N; q += nthr) {
          const double d = (double)ys_s[q];
          chi_s[d0 + q] += d;
          dm = isfinite(d) ? fmax(dm, fabs(d)) : INFINITY;
        }
        dm = block_max(dm, red);
        if (!isfinite(dm)) finite = false;
        dmax = fmax(dmax, dm);
        continue;
      }
      if (b.type != FSI_BODY_TORSIONAL) continue;
      const double sn = b_sn[bi], cs = b_cs[bi];
      double part = 0.0;
      for (int p = b.off + tid; p < b.off + b.n; p += nthr) {
        const double q = (double)(p - b.off) * a.ds;
        part += q * (-sn) * f_s[p] + q * cs * f_s[nb + p];
      }
      const double sf = block_sum(part, red);
      const double gk = kb_s ? kb_s[bi * KB_N + KB_G] : 0.0;  // pseudo-force moment at the iterate
      const double dth = (b_rphi[bi] + gk - b_jac[bi] * b_th[bi] + a.ds * sf) * b_ijac[bi];
      __syncthreads();
      if (tid == 0) {
        b_tp[bi] = b_th[bi];
        b_th[bi] += dth;
        b_ph[bi] = a.two_dt * b_th[bi] - b_rth[bi];
      }
      if (!isfinite(dth)) finite = false;
      dmax = fmax(dmax, fabs(dth));
      __syncthreads();
    }
    if (!finite && blockIdx.x == 0 && tid == 0) dev_set_status(a.status, FSI_ERR_NONFINITE);
    converged = (dmax <= a.tol) || !finite;
    clk.mark(6);
    if (converged) break;
    // No barrier here: shared-memory state is CTA-local; the global K, its float copy and the residual
    // rows are next written after this CTA passes the phase-B barrier of the next iteration, which every
    // CTA reaches only after its last read of them in this iteration.
  }

  // ---- Newmark update, forces, history (CTA 0)
  if (blockIdx.x == 0) {
    // every CTA passed its last barrier of warps 0-3 before the grid barrier that followed it
    if (tid == 0) a.ctrl[15] = 0;
    if (tid == 0 && !converged) dev_set_status(a.status, FSI_ERR_NOT_CONVERGED);
    for (int k = tid; k < nf; k += nthr) a.f[k] = f_s[k];  // surface stress for the corrector
    const int slot = a.ctrl[2] % a.hist_cap;
    // force and moment sums of all bodies, kOs bodies at a time reduced together; a torsional body's S is that of
    // the final solve, whose angle b_tp gave b_sn, b_cs at the start of the last iteration
    constexpr int kOs = 5;
    __shared__ double fsum_s[kMaxBodies][3];
    for (int g0 = 0; g0 < a.n_bodies; g0 += kOs) {
      double part[3 * kOs];
#pragma unroll
      for (int k = 0; k < kOs; ++k) {
        double px = 0.0, py = 0.0, pm = 0.0;
        const int bi = g0 + k;
        if (bi < a.n_bodies) {
          const bool tb = bt_s[bi] == FSI_BODY_TORSIONAL;
          const double sn = tb ? b_sn[bi] : 0.0, cs = tb ? b_cs[bi] : 0.0;
          const int off = boff_s[bi], n = bn_s[bi];
          for (int p = off + tid; p < off + n; p += nthr) {
            const double fxp = f_s[p], fyp = f_s[nb + p];
            const double q = (double)(p - off) * a.ds;
            px += fxp;
            py += fyp;
            pm += q * (-sn) * fxp + q * cs * fyp;
          }
        }
        part[3 * k] = px;
        part[3 * k + 1] = py;
        part[3 * k + 2] = pm;
      }
      block_sum_k<3 * kOs>(part, red);
      if (tid == 0)
#pragma unroll
        for (int k = 0; k < kOs; ++k)
          if (g0 + k < a.n_bodies)
            for (int m = 0; m < 3; ++m) fsum_s[g0 + k][m] = part[3 * k + m];
    }
    __syncthreads();
    for (int bi = 0; bi < a.n_bodies; ++bi) {
      const BodyDev b = a.bodies[bi];
      const double sx = fsum_s[bi][0], sy = fsum_s[bi][1], sm = fsum_s[bi][2];
      double tipd = 0.0, tipr = 0.0;
      if (b.type == FSI_BODY_DEFORMABLE) {
        const int N = b.n - 1, e0 = b.el_off, d0 = 3 * e0;
        for (int q = tid; q < 3 * N; q += nthr) {  // trapezoidal Newmark update to chi_{n+1}
          const int g = d0 + q;
          const double cn = chi_s[g], dc = cn - a.bchi[g], zo = a.bzeta[g];
          a.bzdot[g] = a.four_dt2 * dc - 2.0 * a.two_dt * zo - a.bzdot[g];
          a.bzeta[g] = a.two_dt * dc - zo;
          a.bchi[g] = cn;
        }
        for (int e = tid; e < N; e += nthr) {  // reference chords at chi_{n+1} for the next step
          double xa = b.hx, ya = b.hy;
          if (e > 0) {
            xa = chi_s[d0 + 3 * (e - 1)];
            ya = chi_s[d0 + 3 * (e - 1) + 1];
          }
          const double dx = chi_s[d0 + 3 * e] - xa, dy = chi_s[d0 + 3 * e + 1] - ya;
          const double il = beam::rsqrt_d(fma(dx, dx, dy * dy));
          const double c = dx * il, sc = dy * il;
          double* rf = a.bref + 3 * (e0 + e);
          rf[0] += beam::chord_rotation(rf[1], rf[2], c, sc);
          rf[1] = c;
          rf[2] = sc;
        }
        __syncthreads();
        if (tid == 0) {  // tip displacement normal to the undeformed flag, and its rate
          const int gt = d0 + 3 * (N - 1);
          const double len = (double)N * a.ds;
          tipd = (chi_s[gt] - (b.hx + len * b.ca0)) * (-b.sa0) + (chi_s[gt + 1] - (b.hy + len * b.sa0)) * b.ca0;
          tipr = a.bzeta[gt] * (-b.sa0) + a.bzeta[gt + 1] * b.ca0;
        }
      }
      if (tid == 0) {
        BodyState& s = a.st[bi];
        s.fx = a.ds * sx;
        s.fy = a.ds * sy;
        s.moment = b.type == FSI_BODY_TORSIONAL ? a.ds * sm : 0.0;
        if (b.type == FSI_BODY_TORSIONAL) {
          const double th_new = b_th[bi];
          const double ph_new = a.two_dt * th_new - b_rth[bi];
          s.phidot = a.four_dt2 * (th_new - s.theta) - 2.0 * a.two_dt * s.phi - s.phidot;
          s.theta = th_new;
          s.phi = ph_new;
          s.theta_k = th_new;
          s.phi_k = ph_new;
        } else if (b.type == FSI_BODY_DEFORMABLE) {
          s.theta = tipd;
          s.phi = tipr;
        }
        double* hrow = a.hist + ((long)slot * a.n_bodies + bi) * 6;
        hrow[0] = s.fx;
        hrow[1] = s.fy;
        hrow[2] = s.moment;
        const bool moving = b.type == FSI_BODY_TORSIONAL || b.type == FSI_BODY_DEFORMABLE;
        hrow[3] = moving ? s.theta : 0.0;
        hrow[4] = moving ? s.phi : 0.0;
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
      a.ctrl[12] = refreshes;
    }
    // vertex box that the corrector source (E0^T P^T f, then curl) can touch: cells of the final P, grown
    // by the E0 support (1.5 cells), the hat support (1 cell) and the curl stencil (1 cell)
    int imin = 1 << 30, imax = -1, jmin = 1 << 30, jmax = -1;
    for (int p = tid; p < nb; p += nthr) {
      const int n0 = pidx_s[4 * p];
      if (n0 >= a.n_box) continue;  // appended point: its source is written by its own kernel
      const int ci = pcij_s[2 * p], cj = pcij_s[2 * p + 1];  // hat cell in the (bounding) box
      imin = min(imin, ci);
      imax = max(imax, ci);
      jmin = min(jmin, cj);
      jmax = max(jmax, cj);
    }
    {
      __shared__ int bx[4][8];
      imin = __reduce_min_sync(FULL, imin);
      imax = __reduce_max_sync(FULL, imax);
      jmin = __reduce_min_sync(FULL, jmin);
      jmax = __reduce_max_sync(FULL, jmax);
      if (lane == 0) {
        bx[0][wid] = imin;
        bx[1][wid] = imax;
        bx[2][wid] = jmin;
        bx[3][wid] = jmax;
      }
      __syncthreads();
      for (int w = 0; w < nw; ++w) {
        imin = min(imin, bx[0][w]);
        imax = max(imax, bx[1][w]);
        jmin = min(jmin, bx[2][w]);
        jmax = max(jmax, bx[3][w]);
      }
    }
    if (tid == 0) {
      a.ctrl[8] = a.i_lo + imin - 3;
      a.ctrl[9] = a.i_lo + imax + 4;
      a.ctrl[10] = a.j_lo + jmin - 3;
      a.ctrl[11] = a.j_lo + jmax + 4;
    }
    clk.mark(7);
    clk.flush(a.phase_ns);
  }
}

}  // namespace

static BeamDims beam_dims(const fsi_ctx* c) {
  int nbmax = 0;
  for (const auto& b : c->bodies) nbmax = b.n > nbmax ? b.n : nbmax;
  return BeamDims{c->nd_tot, c->ne_tot, c->nd_max, c->d_kin ? c->n_bodies : 0, nbmax};
}

// Dynamic shared memory of the FSI kernel: the variant with the float inverse in shared memory, or (big) the
// distributed one.
size_t fsi_smem_bytes(const fsi_ctx* c, bool big) { return fsi_layout(c->nf, c->nb, beam_dims(c), big).total; }
size_t fsi_smem_bytes(const fsi_ctx* c) { return fsi_smem_bytes(c, c->fsi_big != 0); }

// dynamic plus static shared memory of a variant of the FSI kernel within the per-block opt-in limit
bool fsi_smem_fits(const fsi_ctx* c, bool big) {
  cudaFuncAttributes fa;
  int dev = 0, optin = 0;
  if (cudaFuncGetAttributes(&fa, big ? k_fsi<true> : k_fsi<false>) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return fsi_smem_bytes(c, big) + fa.sharedSizeBytes <= (size_t)optin;
}

// row stride (floats) of the float nf x nf matrices of the FSI kernel
int fsi_float_ld(int nf) { return fsi_ldx(nf); }

// CTAs of the FSI kernel per SM at this size (0: does not fit)
int fsi_kernel_max_ctas_per_sm(const fsi_ctx* c) {
  const size_t bytes = fsi_smem_bytes(c);
  const bool big = c->fsi_big != 0;
  if (raise_smem_limit(big ? k_fsi<true> : k_fsi<false>, bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, big ? k_fsi<true> : k_fsi<false>, 256, bytes);
  return n;
}

// every CTA owns at most kMaxR rows of the small system (kMaxRB in the distributed variant)
int fsi_min_grid(int nf, bool big) { return big ? (nf + kMaxRB - 1) / kMaxRB : (nf + kMaxR - 1) / kMaxR; }

fsi_status launch_fsi(fsi_ctx* c) {
  FsiArgs a;
  a.s0 = c->s_all;
  a.fp64 = c->prec == FSI_PREC_MIXED ? 2 : (c->fesz == 8 ? 1 : 0);  // type of the level fields
  a.ps = c->ps;
  a.x0 = c->g.x0;
  a.y0 = c->g.y0;
  a.h = c->g.h;
  a.dt = c->g.dt;
  a.ds = c->ds;
  a.U = c->g.uinf[0];
  a.V = c->g.uinf[1];
  a.tol = c->x.tol;
  a.two_dt = 2.0 / c->g.dt;
  a.four_dt2 = 4.0 / (c->g.dt * c->g.dt);
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
  a.T = c->d_T;
  a.part = c->d_part;
  a.ctrl = c->d_ctrl;
  a.phase_ns = c->phase_on ? c->d_phase : nullptr;  // timers only when asked for: they sit in every step
  a.status = c->d_status;
  a.hist = c->d_hist;
  a.hist_cap = c->hist_cap;
  a.n_def = c->n_def;
  a.nd_tot = c->nd_tot;
  a.ne_tot = c->ne_tot;
  a.nd_max = c->nd_max;
  a.nbody_max = beam_dims(c).nbody_max;
  a.bchi = c->d_bchi;
  a.bzeta = c->d_bzeta;
  a.bzdot = c->d_bzdot;
  a.bref = c->d_bref;
  a.G = c->d_G;
  a.Bw = c->Bw;
  a.bw = c->bw;
  a.pcij = c->d_pcij;
  a.kin = c->d_kin;
  a.kin_cap = c->kin_cap > 0 ? c->kin_cap : 1;
  a.nkb = c->d_kin ? c->n_bodies : 0;
  a.n_box = c->n_box;
  a.app_idx = c->n_app > 0 ? c->d_app_idx : nullptr;
  a.app_win = c->d_app_win;
  a.lb_spins = c->wait_spins ? c->wait_spins : (1u << 22);
  a.n_sdb = c->n_sdb > 1 ? c->n_sdb : 1;
  memcpy(a.sdb, c->sdb, sizeof(a.sdb));
  a.sd_map = c->n_sdb > 1 ? c->d_sd_map : nullptr;
  a.dvec = c->d_dvec;
  a.rsum = c->d_rsum;
  a.resf = c->d_resf;
  const bool big = c->fsi_big != 0;
  a.lb_missing = c->wait_missing;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->fsi_grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = fsi_smem_bytes(c);
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  FSI_CUDA_TRY(raise_smem_limit(big ? k_fsi<true> : k_fsi<false>, cfg.dynamicSmemBytes));
  prof_mark(c, KC_FSI);
  FSI_CUDA_TRY(cudaLaunchKernelEx(&cfg, big ? k_fsi<true> : k_fsi<false>, a));
  prof_mark(c, KC_FSI);
  c->launches_per_step += 1;
  return FSI_OK;
}
