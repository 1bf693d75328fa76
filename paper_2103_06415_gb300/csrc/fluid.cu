// Fluid part of one time step on the nested levels: advection + right-hand side (App. A, AB2/CN),
// multidomain coupling (Sec. 5, far-field multidomain), the DST-diagonalised predictor solves
// (Eq. predictor2) and the corrector (Eq. corrector2) with its surface-stress source.
#include <cstdio>
#include <mutex>
#include <type_traits>
#include "spec.cuh"

namespace {

// ---------------------------------------------------------------------------------------------
// Launch shapes of the FFT passes for a length L = r3 * 2^logP: 4 * PER * threads = nf * 2^logP (nf
// transforms per CTA).  Lengths 3 * 2^k stop at 3072 (grids of 1536 cells), so they always take PER = 1.
struct FftCfg {
  int nthr, per, nf, r3, logP, L;
};
FftCfg fft_cfg(int logP, int r3) {
  const int P = 1 << logP;
  FftCfg c;
  c.nthr = P / 4;
  if (c.nthr < 32) c.nthr = 32;
  if (c.nthr > 256) c.nthr = 256;
  c.per = 1;
  while (4 * c.per * c.nthr < P) c.per *= 2;
  c.nf = 4 * c.per * c.nthr / P;
  c.r3 = r3;
  c.logP = logP;
  c.L = r3 << logP;
  return c;
}

// Calls LAUNCH(PER, R3) with the template arguments of a launch shape.
#define FFT_DISPATCH(cfg, LAUNCH)                     \
  do {                                                \
    if ((cfg).r3 == 3) {                              \
      LAUNCH(1, 3);                                   \
    } else if ((cfg).per == 1) {                      \
      LAUNCH(1, 1);                                   \
    } else if ((cfg).per == 2) {                      \
      LAUNCH(2, 1);                                   \
    } else {                                          \
      LAUNCH(4, 1);                                   \
    }                                                 \
  } while (0)

template <typename T, typename TF>
void set_smem_limits_once();

template <typename T, typename TF = T>
void set_smem_limits() {
  static std::once_flag once;  // contexts may run on several host threads (the server's worker)
  std::call_once(once, set_smem_limits_once<T, TF>);
}

template <typename T, typename TF>
void set_smem_limits_once() {
  const int big = 200 * 1024;
  cudaFuncSetAttribute(dst::k_xf<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xf<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xf<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_ysolve<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_ysolve<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_ysolve<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xi<T, 1, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xi<T, 2, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xi<T, 4, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xf<T, 1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_ysolve<T, 1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if constexpr (std::is_same<T, float>::value) {
    cudaFuncSetAttribute(dst::k_ysolve<T, 1, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(dst::k_ysolve<T, 2, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(dst::k_ysolve<T, 4, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(dst::k_ysolve<T, 1, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  }
  cudaFuncSetAttribute(dst::k_xi<T, 1, TF, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

// ---------------------------------------------------------------------------------------------
// O2: advection N = div(u w) with vertex-averaged velocities (reading R7) and
// rhs = w/dt + lap_h w/(2 Re) - 3/2 N^n + 1/2 N^{n-1}.  Block (32, 8) = one tile of interior vertices; the
// tile of w and s with a one-vertex halo is staged in shared memory (each value read once from L2).
// Per-level constants in the transform precision T (computed on the host).  The fields are of type TF
// (TF = T, or double fields with float transforms in the mixed mode: the differences of field values are
// taken in TF, the rest in T).  delta: every level takes the right-hand side of the increment w* - w~^n
// instead, A_w (w* - w~^n) = lap_h w~^n / Re - 3/2 N^n + 1/2 N^{n-1} (the same equation with
// A_w w~^n = w~^n/dt - lap_h w~^n/(2 Re) moved to the right; its boundary values are the ring increments),
// computed in TF throughout, where w~^n is the level's vorticity with the finer levels' values injected at
// the vertices they cover.  The injected values are written into the level's own array, so that the
// increment is added to w~^n, and the defect w~^n + lap_h s^n of the level's streamfunction goes to its
// slot of `defect` (levels lvl apart).
template <typename T>
struct RhsConst {
  T i2h[12], inv_h2[12];  // 1/(2 h_g), 1/h_g^2 for level g (at most 12 levels)
  T inv_dt, half_inv_re, inv_re, U, V;
  float ih2_hi[12], ih2_lo[12];  // 1/h_g^2 as a float pair, for the defect of the increment form
};

template <typename T, typename TF = T>
__global__ void __launch_bounds__(256) k_rhs(TF* __restrict__ w_all, const TF* __restrict__ s_all,
                                             T* __restrict__ np_all, T* __restrict__ rhs_all, long lvl, long ps,
                                             int nx, int ny, RhsConst<T> k, int first, int delta,
                                             T* __restrict__ defect) {
  pdl_enter();
  __shared__ TF tw[10][35], ts[10][35];
  const int g = blockIdx.z;
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8;  // tile vertex (i0 + 1, j0 + 1) at smem (1, 1)
  const TF* s = s_all + (long)g * lvl;
  TF* w_own = w_all + (long)g * lvl;
  const int t = threadIdx.y * 32 + threadIdx.x;
  const int i = i0 + threadIdx.x + 1, j = j0 + threadIdx.y + 1;
  const bool inner = i < nx && j < ny;
  const long o = (long)j * ps + i;
  T* np = np_all + (long)g * lvl;
  // every global load of the thread is issued before any is consumed: N^{n-1} of its vertex and its (at
  // most two) elements of the 10 x 34 tile of w and s
  const T nprev = (inner && !first) ? T(np[o]) : T(0);
  TF wv[2], sv[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int e = t + 256 * q;
    const int r = e / 34, c = e - r * 34;
    const int I = i0 + c, J = j0 + r;  // vertex indices 0..nx, 0..ny
    wv[q] = sv[q] = TF(0);
    if (e < 10 * 34 && I <= nx && J <= ny) {
      // O1 on the fly: a vertex strictly inside a finer level takes the vorticity of the finest level that
      // contains it (the coarse array itself is overwritten by this level's solve before any other use)
      int gi = g, ii = I, jj = J;
      while (gi > 0 && abs(2 * ii - nx) < nx / 2 && abs(2 * jj - ny) < ny / 2) {
        ii = 2 * ii - nx / 2;
        jj = 2 * jj - ny / 2;
        --gi;
      }
      wv[q] = w_all[(long)gi * lvl + (long)jj * ps + ii];
      sv[q] = s[(long)J * ps + I];
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int e = t + 256 * q;
    if (e < 10 * 34) {
      const int r = e / 34, c = e - r * 34;
      tw[r][c] = wv[q];
      ts[r][c] = sv[q];
    }
  }
  __syncthreads();
  if (!inner) return;
  const int x = threadIdx.x + 1, y = threadIdx.y + 1;
  const long oi = (long)(j - 1) * ps + (i - 1);
  if constexpr (std::is_same<TF, f2s>::value) {
    if (delta) {
      // The increment right-hand side: the differences of field values, which cancel, as exact float pairs,
      // then rounded to float; the products and sums of those differences in float.  The flux differences are
      // rewritten so that no product of two field values is differenced: ue we - uw ww = ue (we - wc) -
      // uw (ww - wc) + (ue - uw) wc, with ue - uw a second difference of s summed in pairs.
      const T i2h = k.i2h[g], ih2 = k.inv_h2[g];
      const TF wc = tw[y][x];
      const TF dwe = tw[y][x + 1] - wc, dww = tw[y][x - 1] - wc, dwn = tw[y + 1][x] - wc, dws = tw[y - 1][x] - wc;
      const TF lapd = (dwe + dww) + (dwn + dws);
      const TF sne = ts[y + 1][x + 1], sse = ts[y - 1][x + 1], snw = ts[y + 1][x - 1], ssw = ts[y - 1][x - 1];
      const TF dse = sne - sse, dsw = snw - ssw, dsn = sne - snw, dss = sse - ssw;
      const T ue = T(dse) * i2h + k.U, uw = T(dsw) * i2h + k.U;
      const T vn = -T(dsn) * i2h + k.V, vs = -T(dss) * i2h + k.V;
      const T du = T(dse - dsw) * i2h, dv = -T(dsn - dss) * i2h;  // ue - uw, vn - vs
      const T wcf = T(wc);
      const T fx = ue * T(dwe) - uw * T(dww) + du * wcf;
      const T fy = vn * T(dwn) - vs * T(dws) + dv * wcf;
      const T n = (fx + fy) * i2h;
      const T nold = first ? n : np[o];
      np[o] = n;
      const long og = (long)g * lvl;
      rhs_all[og + oi] = T(lapd) * ih2 * k.inv_re - T(1.5) * n + T(0.5) * nold;
      // defect of the streamfunction (a small difference, in pairs, with 1/h^2 as a pair): the increment of s
      // solves -lap_h ds = dw + defect, so s* satisfies -lap_h s* = w* to the rounding of the increment (the
      // rounding of earlier float transforms left in s is removed at every step instead of accumulating)
      const TF sc = ts[y][x];
      const TF laps = ((ts[y][x + 1] - sc) + (ts[y][x - 1] - sc)) + ((ts[y + 1][x] - sc) + (ts[y - 1][x] - sc));
      const float p = laps.hi * k.ih2_hi[g];
      const TF lap_s = f2s_norm(p, fmaf(laps.hi, k.ih2_hi[g], -p) + (laps.hi * k.ih2_lo[g] + laps.lo * k.ih2_hi[g]));
      defect[og + oi] = T(wc + lap_s);
      // w~^n into the level's array at a covered vertex (no launch reads a level's covered vertices: they
      // are always taken from the finest level that contains them)
      if (g > 0 && abs(2 * i - nx) < nx / 2 && abs(2 * j - ny) < ny / 2) w_own[o] = wc;
      return;
    }
  }
  const T i2h = k.i2h[g];
  const TF wc = tw[y][x], we = tw[y][x + 1], ww = tw[y][x - 1], wn = tw[y + 1][x], wsx = tw[y - 1][x];
  // ubar at (i+-1, j) = (s[j+1] - s[j-1])/(2h) + U ; vbar at (i, j+-1) = -(s[i+1] - s[i-1])/(2h) + V
  const T ue = T(ts[y + 1][x + 1] - ts[y - 1][x + 1]) * i2h + k.U;
  const T uw = T(ts[y + 1][x - 1] - ts[y - 1][x - 1]) * i2h + k.U;
  const T vn = -T(ts[y + 1][x + 1] - ts[y + 1][x - 1]) * i2h + k.V;
  const T vs = -T(ts[y - 1][x + 1] - ts[y - 1][x - 1]) * i2h + k.V;
  const T n = (ue * T(we) - uw * T(ww)) * i2h + (vn * T(wn) - vs * T(wsx)) * i2h;
  T lap;
  if constexpr (std::is_same<TF, f2s>::value)
    lap = T(((we - wc) + (ww - wc)) + ((wn - wc) + (wsx - wc))) * k.inv_h2[g];
  else
    lap = T(we + ww + wn + wsx - TF(4) * wc) * k.inv_h2[g];
  const T nold = first ? n : nprev;
  np[o] = n;
  const T base = T(wc) * k.inv_dt + lap * k.half_inv_re;
  rhs_all[(long)g * lvl + oi] = base - T(1.5) * n + T(0.5) * nold;
}

// O3 and the boundary-side transforms of a nested level in one launch.  Ring vectors: side 0 = left/right
// columns (j = 1..ny-1) of w then s, side 1 = bottom/top rows (i = 1..nx-1) of w then s.  A block takes a
// group of vectors of one side, computes them from the coarse level (injection at coincident vertices,
// midpoint average otherwise; reading R5), writes them into the
// fine level's boundary ring and their unnormalised DST-I into the ring spectra (8 x ring_ld: wL wR wB wT
// sL sR sB sT).  Block 0 also writes the eight corner values.  blockDim = 256, 4 PER 256 = nf L per block.
template <typename T>
__device__ __forceinline__ T ring_value(const T* __restrict__ c, long ps, int nx, int ny, int i, int j) {
  const int a = i + nx / 2, b = j + ny / 2;
  const int I0 = a >> 1, J0 = b >> 1;
  const int I1 = I0 + (a & 1), J1 = J0 + (b & 1);
  return field_mid(c[(long)J0 * ps + I0], c[(long)J1 * ps + I1]);
}

// delta: the spectra are those of the ring increments (new value minus the fine level's current one; the
// increment form of the finest level in the mixed mode).  TF: type of the level fields.
// Side transform lengths: x (side 1) R3X * 2^logPx, y (side 0) R3Y * 2^logPy; per side a CTA transforms
// nf = 4 PER blockDim / 2^logP vectors.
template <typename T, int PER, typename TF = T, int R3X = 1, int R3Y = 1>
__global__ void __launch_bounds__(256) k_ring_dst(TF* __restrict__ wf, TF* __restrict__ sf, const TF* __restrict__ wc,
                                                  const TF* __restrict__ sc, long ps, int nx, int ny,
                                                  T* __restrict__ ring, long ring_ld,
                                                  const typename C2<T>::t* __restrict__ twx,
                                                  const typename C2<T>::t* __restrict__ twy, int logLx, int logLy,
                                                  int nblk_y, int delta) {
  pdl_enter();
  using c2 = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2* buf = reinterpret_cast<c2*>(smem_raw);
  const int side = (int)blockIdx.x < nblk_y ? 0 : 1;
  const int logL = side ? logLx : logLy, L = (side ? R3X : R3Y) << logL;
  const int N = side ? nx - 1 : ny - 1;
  const int nf = 4 * PER * (int)blockDim.x / (1 << logL);
  const int v0 = 2 * nf * (side ? (int)blockIdx.x - nblk_y : (int)blockIdx.x);
  if (blockIdx.x == 0 && threadIdx.x < 8) {  // corners (i, j) in {0, nx} x {0, ny} of w and s
    const int q = threadIdx.x & 3;
    const int i = (q & 1) ? nx : 0, j = (q & 2) ? ny : 0;
    if (threadIdx.x < 4) wf[(long)j * ps + i] = ring_value(wc, ps, nx, ny, i, j);
    else sf[(long)j * ps + i] = ring_value(sc, ps, nx, ny, i, j);
  }
  const c2* tws =
      dst::stage_twiddles<T>(buf + (long)nf * L, side ? twx : twy, L, ((size_t)nf * L + L) * sizeof(c2));
  dst::zero_ends<T>(buf, nf, L);
  // The gather of the coarse values (two per ring vertex, and the fine level's current value for an increment):
  // a thread's loads for four of its vertices are issued before any is used (with only a few CTAs in the
  // launch, one vertex at a time left the kernel waiting on one load after another).
  constexpr int U = 4;
  for (int idx0 = threadIdx.x; idx0 < nf * N; idx0 += blockDim.x * U) {
    TF c0[U][2], c1[U][2], fo[U][2];
    int fo_off[U][2];  // offset of the fine vertex; -1 where the vector does not exist
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = idx0 + u * (int)blockDim.x;
      const int f = idx / N, n = idx - f * N;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int v = v0 + 2 * f + e;
        fo_off[u][e] = -1;
        if (idx < nf * N && v < 4) {
          const int i = side ? n + 1 : ((v & 1) ? nx : 0);
          const int j = side ? ((v & 1) ? ny : 0) : n + 1;
          const TF* c = v < 2 ? wc : sc;
          const int ia = i + nx / 2, jb = j + ny / 2;
          const int I0 = ia >> 1, J0 = jb >> 1, I1 = I0 + (ia & 1), J1 = J0 + (jb & 1);
          c0[u][e] = c[(long)J0 * ps + I0];
          c1[u][e] = c[(long)J1 * ps + I1];
          fo_off[u][e] = j * (int)ps + i;
          fo[u][e] = delta ? (v < 2 ? wf : sf)[fo_off[u][e]] : TF(0);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = idx0 + u * (int)blockDim.x;
      if (idx >= nf * N) break;
      const int f = idx / N, n = idx - f * N;
      T ab[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        ab[e] = T(0);
        if (fo_off[u][e] >= 0) {
          const TF val = field_mid(c0[u][e], c1[u][e]);  // injection at coincident vertices: c0 == c1
          ab[e] = delta ? T(val - fo[u][e]) : T(val);
          (v0 + 2 * f + e < 2 ? wf : sf)[fo_off[u][e]] = val;
        }
      }
      dst::put_pair<T>(buf + (long)f * L, L, n, ab[0], ab[1]);
    }
  }
  __syncthreads();
  if (side) dst::block_fft<T, PER, R3X>(buf, L, logL, tws);
  else dst::block_fft<T, PER, R3Y>(buf, L, logL, tws);
  const int dmap[2][4] = {{0, 1, 4, 5}, {2, 3, 6, 7}};
  for (int idx = threadIdx.x; idx < nf * N; idx += blockDim.x) {
    const int f = idx / N, n = idx - f * N;
    const int va = v0 + 2 * f;
    const c2 z = buf[(long)f * L + n + 1];
    if (va < 4) ring[dmap[side][va] * ring_ld + n] = T(-0.5) * z.y;
    if (va + 1 < 4) ring[dmap[side][va + 1] * ring_ld + n] = T(0.5) * z.x;
  }
}

// O5 source: src = (ds/h^2) curl_h(E0^T P^T f) on the level-0 vertices near the body.  Deterministic
// gather (no atomics): every vertex sums the contributions of the body points in point order, so a run
// gives the same bits every time.
//
// Face weights of one body point with hat cell (ci, cj) and hat weights w_ab (node (ci + a, cj + b)):
// E0 puts a u-value at vertex (vi, vj) on the u-faces (vi + d, vj +- 1/2) with weight wx3(d) / 2,
// wx3 = (1/6, 2/3, 1/6), and a v-value on the v-faces (vi +- 1/2, vj + d) likewise.  With
//   U_b(d) = sum_a w_ab wx3(d - a)   and   V_a(e) = sum_b w_ab wx3(e - b),   d, e in -1..2,
// the u-face (i, j + 1/2) receives (1/2) sum_{b : j - cj - b in {-1, 0}} U_b(i - ci) fx and the v-face
// (i + 1/2, j) receives (1/2) sum_{a : i - ci - a in {-1, 0}} V_a(j - cj) fy.  The tables are built once
// per point (times the stress) in shared memory.
template <typename T>
__device__ __forceinline__ T wx3t(int d) { return d == 0 ? T(2.0 / 3.0) : ((d == 1 || d == -1) ? T(1.0 / 6.0) : T(0)); }

struct SrcPoint {
  int ci, cj;
};

// u-face (fi, fj + 1/2) value of point p (tables ut[b][d + 1] = U_b(d) fx / 2)
template <typename T>
__device__ __forceinline__ T u_face(const T* ut, int ci, int cj, int fi, int fj) {
  const int d = fi - ci;
  if (d < -1 || d > 2) return T(0);
  T v = T(0);
  const int e = fj - cj;  // b with e - b in {-1, 0}: b = e or b = e + 1
  if (e == 0 || e == 1) v += ut[e * 4 + d + 1];
  if (e == -1 || e == 0) v += ut[(e + 1) * 4 + d + 1];
  return v;
}
// v-face (fi + 1/2, fj) value of point p (tables vt[a][e + 1] = V_a(e) fy / 2)
template <typename T>
__device__ __forceinline__ T v_face(const T* vt, int ci, int cj, int fi, int fj) {
  const int e = fj - cj;
  if (e < -1 || e > 2) return T(0);
  T v = T(0);
  const int d = fi - ci;
  if (d == 0 || d == 1) v += vt[d * 4 + e + 1];
  if (d == -1 || d == 0) v += vt[(d + 1) * 4 + e + 1];
  return v;
}

// Thread per vertex over tiles of 32 x 4 vertices covering the Omega_0 box grown by 3 cells.  Vertices
// outside the box written by the FSI kernel (ctrl[8..11]) are set to zero.  A tile that meets the box
// walks the points in chunks of kSrcChunk and keeps, in point order, those whose face support can reach
// it, with their face tables.  The face values and the curl are taken in TS and stored in T: along a plate
// the normal stress is smooth, so the curl is a small difference of large face values (about h / chord of
// them), and the mixed mode takes it in double so that only the transform of the source is in float.
constexpr int kSrcChunk = 256;

template <typename T, typename TS = T>
__global__ void __launch_bounds__(128) k_src(T* __restrict__ src, long ps, int nx, int ny, const int* __restrict__ pidx,
                                             const int* __restrict__ pcij,
                                             const double* __restrict__ pw, const double* __restrict__ f, int nb, int ni,
                                             int i_lo, int i_hi, int j_lo, int j_hi, const int* __restrict__ box,
                                             TS coef, int n_box) {
  pdl_enter();
  __shared__ TS tab[kSrcChunk * 16];  // [chunk point][16]: ut (8) then vt (8)
  __shared__ SrcPoint pt[kSrcChunk];
  __shared__ int wcount[4], n_sel;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ti0 = i_lo - 3 + blockIdx.x * 32, tj0 = j_lo - 3 + blockIdx.y * 4;
  const int i = ti0 + lane, j = tj0 + wid;
  const int bi0 = box[0], bi1 = box[1], bj0 = box[2], bj1 = box[3];
  const bool tile_hits = ti0 <= bi1 && ti0 + 31 >= bi0 && tj0 <= bj1 && tj0 + 3 >= bj0;  // block-uniform
  const bool valid = i >= 1 && i <= nx - 1 && i <= i_hi + 3 && j >= 1 && j <= ny - 1 && j <= j_hi + 3;
  const bool inside = i >= bi0 && i <= bi1 && j >= bj0 && j <= bj1;
  if (valid && !inside) src[(long)(j - 1) * ps + (i - 1)] = T(0);
  if (!tile_hits) return;
  TS fve = 0, fvw = 0, fun = 0, fus = 0;
  for (int c0 = 0; c0 < nb; c0 += kSrcChunk) {
    const int c1 = c0 + kSrcChunk < nb ? c0 + kSrcChunk : nb;
    // select the chunk's points whose faces enter the curl at some vertex of this tile: vertex offsets
    // i - ci and j - cj in -1..2
    if (tid == 0) n_sel = 0;
    __syncthreads();
    for (int base = c0; base < c1; base += 128) {
      const int p = base + tid;
      int ci = 0, cj = 0;
      bool take = false;
      if (p < c1) {
        const int n0 = pidx[4 * p];
        ci = pcij[2 * p] + i_lo;  // hat cell in the (bounding) box, as grid vertex indices
        cj = pcij[2 * p + 1] + j_lo;
        take = n0 < n_box && ci - 1 <= ti0 + 31 && ci + 2 >= ti0 && cj - 1 <= tj0 + 3 && cj + 2 >= tj0;  // appended: elsewhere
      }
      const unsigned m = __ballot_sync(0xffffffffu, take);
      if (lane == 0) wcount[wid] = __popc(m);
      __syncthreads();
      int off = n_sel;
      for (int w = 0; w < wid; ++w) off += wcount[w];
      if (take) {
        const int q = off + __popc(m & ((1u << lane) - 1u));
        pt[q].ci = ci;
        pt[q].cj = cj;
        const TS w00 = TS(pw[4 * p]), w10 = TS(pw[4 * p + 1]), w01 = TS(pw[4 * p + 2]), w11 = TS(pw[4 * p + 3]);
        const TS fx = TS(0.5) * TS(f[p]), fy = TS(0.5) * TS(f[nb + p]);
        TS* t = tab + 16 * q;
        for (int d = -1; d <= 2; ++d) {
          t[0 * 4 + d + 1] = (w00 * wx3t<TS>(d) + w10 * wx3t<TS>(d - 1)) * fx;  // U_0(d)
          t[1 * 4 + d + 1] = (w01 * wx3t<TS>(d) + w11 * wx3t<TS>(d - 1)) * fx;  // U_1(d)
          t[8 + 0 * 4 + d + 1] = (w00 * wx3t<TS>(d) + w01 * wx3t<TS>(d - 1)) * fy;  // V_0(e = d)
          t[8 + 1 * 4 + d + 1] = (w10 * wx3t<TS>(d) + w11 * wx3t<TS>(d - 1)) * fy;  // V_1(e = d)
        }
      }
      __syncthreads();
      if (tid == 0) n_sel += wcount[0] + wcount[1] + wcount[2] + wcount[3];
      __syncthreads();
    }
    const int ns = n_sel;
    if (valid && inside) {
      for (int q = 0; q < ns; ++q) {
        const int ci = pt[q].ci, cj = pt[q].cj;
        if (i < ci - 1 || i > ci + 2 || j < cj - 1 || j > cj + 2) continue;
        const TS* t = tab + 16 * q;
        fun += u_face<TS>(t, ci, cj, i, j);
        fus += u_face<TS>(t, ci, cj, i, j - 1);
        fve += v_face<TS>(t + 8, ci, cj, i, j);
        fvw += v_face<TS>(t + 8, ci, cj, i - 1, j);
      }
    }
    __syncthreads();  // the next chunk overwrites the tables
  }
  if (!valid || !inside) return;
  // curl at (i,j): (Fv(i+1/2,j) - Fv(i-1/2,j))/h - (Fu(i,j+1/2) - Fu(i,j-1/2))/h
  src[(long)(j - 1) * ps + (i - 1)] = T(coef * ((fve - fvw) - (fun - fus)));
}

// ---------------------------------------------------------------------------------------------
// Pass p of the sine transforms runs as a tensor-core GEMM (FP32 contexts that chose it; dst_gemm.cu).
template <typename T>
bool use_gemm(const fsi_ctx* c, int p) {
  return std::is_same<T, float>::value && c->gd && c->dst_gemm[p];
}

// Pass XF of nlev levels in one launch (blockIdx.y = level): right-hand sides lvl_elems apart, x-transforms
// to the scratch slots T1 + level * Nx * ldT.  The tensor-core variant takes one level.
template <typename T>
fsi_status xf_pass(fsi_ctx* c, const T* rhs, int nlev) {
  using c2 = typename C2<T>::t;
  set_smem_limits<T>();
  const FftCfg cx = fft_cfg(c->logPx, c->r3x);
  const int Lx = cx.L;
  const c2* twx = (const c2*)c->twx;
  prof_mark(c, KC_XF);
  if (use_gemm<T>(c, 0)) {
    if (nlev != 1) return FSI_ERR_UNSUPPORTED;  // one level per tensor-core pass
    const fsi_status st = gemm_xf(c, (const float*)rhs);
    if (st != FSI_OK) return st;
  } else {
    dim3 grid((c->Ny + 2 * cx.nf - 1) / (2 * cx.nf), nlev);
    const size_t sm = dst::pass_smem<T>((size_t)cx.nf * Lx, Lx);
    const long ib = c->lvl_elems, ob = (long)c->Nx * c->ldT;
#define XF_LAUNCH(P, R) FSI_CUDA_TRY(pdl_launch(dst::k_xf<T, P, R>, grid, dim3(cx.nthr), sm, c->stream, rhs, c->ps, ib, c->Ny, c->Nx, (T*)c->T1, c->ldT, ob, twx, cx.logP, cx.nf))
    FFT_DISPATCH(cx, XF_LAUNCH);
#undef XF_LAUNCH
  }
  prof_mark(c, KC_XF);
  c->launches_per_step += 1;
  return FSI_OK;
}

// Pass Y of level g (spacing h 2^g) from the x-transforms at t1, with the ring spectra when use_ring, and
// the x-transforms t1r of the streamfunction defect when not null (float transforms only).
template <typename T>
fsi_status y_pass(fsi_ctx* c, int g, const T* t1, int use_ring, const T* t1r = nullptr) {
  using c2 = typename C2<T>::t;
  set_smem_limits<T>();
  const FftCfg cy = fft_cfg(c->logPy, c->r3y);
  const int Ly = cy.L;
  const c2* twy = (const c2*)c->twy;
  prof_mark(c, KC_YSOLVE);
  const double h = c->g.h * (double)(1 << g);
  const dst::SpecParams<T> sp = spec_params<T>(c, h, use_ring ? (const T*)c->ring : nullptr);
  if (use_gemm<T>(c, 1)) {
    if (t1 != (const T*)c->T1) return FSI_ERR_UNSUPPORTED;  // the tensor-core pass reads slot 0
    if constexpr (std::is_same<T, float>::value) {
      const fsi_status st = gemm_ysolve(c, sp);
      if (st != FSI_OK) return st;
    }
  } else {
    dim3 grid((c->Nx + 2 * cy.nf - 1) / (2 * cy.nf), 1);
    if (t1r) {
      if constexpr (std::is_same<T, float>::value) {
        const size_t sm = dst::pass_smem<T>((size_t)2 * cy.nf * Ly, Ly);
#define Y_LAUNCH(P, R) FSI_CUDA_TRY(pdl_launch(dst::k_ysolve<T, P, R, true>, grid, dim3(cy.nthr), sm, c->stream, t1, c->ldT, 0, c->Nx, c->Ny, (T*)c->T2w, (T*)c->T2s, c->ldX, 0, twy, cy.logP, cy.nf, sp, t1r))
        FFT_DISPATCH(cy, Y_LAUNCH);
#undef Y_LAUNCH
      } else {
        return FSI_ERR_UNSUPPORTED;
      }
    } else {
      const size_t sm = dst::pass_smem<T>((size_t)2 * cy.nf * Ly, Ly);
#define Y_LAUNCH(P, R) FSI_CUDA_TRY(pdl_launch(dst::k_ysolve<T, P, R>, grid, dim3(cy.nthr), sm, c->stream, t1, c->ldT, 0, c->Nx, c->Ny, (T*)c->T2w, (T*)c->T2s, c->ldX, 0, twy, cy.logP, cy.nf, sp, (const T*)nullptr))
      FFT_DISPATCH(cy, Y_LAUNCH);
#undef Y_LAUNCH
    }
  }
  prof_mark(c, KC_YSOLVE);
  c->launches_per_step += 1;
  return FSI_OK;
}

// Pass XI into the level fields w, s of type TF (mode 0 store, 1 subtract, 2 add): 2*nf rows of one field
// per CTA, rows j, j+1 sharing one FFT.
template <typename T, typename TF = T>
fsi_status xi_pass(fsi_ctx* c, TF* w, TF* s, int mode) {
  using c2 = typename C2<T>::t;
  set_smem_limits<T, TF>();
  const FftCfg cx = fft_cfg(c->logPx, c->r3x);
  const int Lx = cx.L;
  const c2* twx = (const c2*)c->twx;
  prof_mark(c, KC_XI);
  if (use_gemm<T>(c, 2)) {
    if constexpr (std::is_same<T, TF>::value) {
      if (mode == 2) return FSI_ERR_UNSUPPORTED;
      const fsi_status st = gemm_xi(c, (float*)w, (float*)s, mode);
      if (st != FSI_OK) return st;
    } else {
      return FSI_ERR_UNSUPPORTED;
    }
  } else {
    dim3 grid(dst::xi_blocks(c->Ny, cx.nf), 1);
    const size_t sm = dst::pass_smem<T>((size_t)cx.nf * Lx, Lx);
#define XI_LAUNCH(P, R) FSI_CUDA_TRY(pdl_launch(dst::k_xi<T, P, TF, R>, grid, dim3(cx.nthr), sm, c->stream, (const T*)c->T2w, (const T*)c->T2s, c->ldX, 0, c->Ny, c->Nx, w, s, c->ps, 0, mode, twx, cx.logP, cx.nf))
    FFT_DISPATCH(cx, XI_LAUNCH);
#undef XI_LAUNCH
  }
  prof_mark(c, KC_XI);
  FSI_CUDA_TRY(cudaGetLastError());
  c->launches_per_step += 1;
  return FSI_OK;
}

template <typename T, typename TF = T>
fsi_status level_solve_t(fsi_ctx* c, int g, const T* rhs, TF* w, TF* s, int use_ring, int mode) {
  fsi_status st = xf_pass<T>(c, rhs, 1);
  if (st == FSI_OK) st = y_pass<T>(c, g, (const T*)c->T1, use_ring);
  if (st == FSI_OK) st = xi_pass<T, TF>(c, w, s, mode);
  return st;
}

template <typename T, typename TF = T>
fsi_status ring_spectra_t(fsi_ctx* c, int g, int delta) {
  using c2 = typename C2<T>::t;
  TF* wf = (TF*)c->w_all + (long)g * c->lvl_elems;
  TF* sf = (TF*)c->s_all + (long)g * c->lvl_elems;
  const TF* wc = (const TF*)c->w_all + (long)(g + 1) * c->lvl_elems;
  const TF* sc = (const TF*)c->s_all + (long)(g + 1) * c->lvl_elems;
  // per side nf = 4 PER 256 / 2^logP vectors per CTA; grids with a 3 * 2^k axis keep both power-of-two parts
  // at most 1024 (checked at fsi_create), so they take PER = 1
  const int Pmax = 1 << (c->logPx > c->logPy ? c->logPx : c->logPy);
  const int per = Pmax <= 1024 ? 1 : Pmax / 1024;
  const int nf_y = 4 * per * 256 / (1 << c->logPy), nf_x = 4 * per * 256 / (1 << c->logPx);
  const int nblk_y = (4 + 2 * nf_y - 1) / (2 * nf_y), nblk_x = (4 + 2 * nf_x - 1) / (2 * nf_x);
  const int Lx = c->r3x << c->logPx, Ly = c->r3y << c->logPy;
  const int r3max = c->r3x > c->r3y ? c->r3x : c->r3y;
  const size_t sm = dst::pass_smem<T>((size_t)4 * per * 256 * r3max, Lx > Ly ? Lx : Ly);
  const c2* twx = (const c2*)c->twx;
  const c2* twy = (const c2*)c->twy;
  static std::once_flag attrs;  // per instantiation; contexts may run on several host threads
  std::call_once(attrs, [] {
    cudaFuncSetAttribute(k_ring_dst<T, 1, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_ring_dst<T, 2, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_ring_dst<T, 4, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_ring_dst<T, 1, TF, 3, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_ring_dst<T, 1, TF, 3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_ring_dst<T, 1, TF, 1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  prof_mark(c, KC_RING);
  const dim3 grid(nblk_y + nblk_x);
#define RING_LAUNCH(P, RX, RY) FSI_CUDA_TRY(pdl_launch(k_ring_dst<T, P, TF, RX, RY>, grid, dim3(256), sm, c->stream, wf, sf, wc, sc, c->ps, c->nx, c->ny, (T*)c->ring, c->ring_ld, twx, twy, c->logPx, c->logPy, nblk_y, delta))
  if (c->r3x == 3 && c->r3y == 3) RING_LAUNCH(1, 3, 3);
  else if (c->r3x == 3) RING_LAUNCH(1, 3, 1);
  else if (c->r3y == 3) RING_LAUNCH(1, 1, 3);
  else if (per == 1) RING_LAUNCH(1, 1, 1);
  else if (per == 2) RING_LAUNCH(2, 1, 1);
  else RING_LAUNCH(4, 1, 1);
#undef RING_LAUNCH
  prof_mark(c, KC_RING);
  c->launches_per_step += 1;
  FSI_CUDA_TRY(cudaGetLastError());
  return FSI_OK;
}

// Predictor of every level, coarse to fine.  In the mixed mode (double fields, float transforms) every level
// is advanced in increment form after the first step: its right-hand side, ring spectra and inverse
// transforms are those of w* - w~^n and s* - s^n, added to the double fields, so the float transforms carry
// errors relative to the increments (O(dt) smaller than the fields) and the fields keep double precision
// (in the full form the float rounding of w^n/dt, which dominates the right-hand side, would accumulate in
// the coarse levels' vorticity step after step).  The increment of s solves
// -lap_h (s* - s^n) = w* - w~^n + (w~^n + lap_h s^n): the defect term is zero for the finest level in exact
// arithmetic and equals the injection's change of w on a coarser one; carrying it makes s* satisfy
// -lap_h s* = w* to float rounding of the increment, so the white rounding noise of earlier float
// transforms does not stay in s (differentiated for the body-point velocities it would be amplified by the
// inverse of the small system).  The first step, and any step after fields were set, takes the full form.
template <typename T, typename TF = T>
fsi_status predictor_t(fsi_ctx* c, int first) {
  TF* w_all = (TF*)c->w_all;
  TF* s_all = (TF*)c->s_all;
  const int delta = (!std::is_same<T, TF>::value && !first) ? 1 : 0;
  // the streamfunction defects of the levels sit in the right-hand-side slots after the last level
  T* defect = delta ? (T*)c->rhs_all + (long)c->G * c->lvl_elems : nullptr;
  {
    dim3 b(32, 8), gr((c->Nx + 31) / 32, (c->Ny + 7) / 8, c->G);
    c->launches_per_step += 1;
    prof_mark(c, KC_RHS);
    RhsConst<T> k = {};
    for (int g = 0; g < c->G; ++g) {
      const double hg = c->g.h * (double)(1 << g);
      k.i2h[g] = T(0.5 / hg);
      k.inv_h2[g] = T(1.0 / (hg * hg));
      const f2s ih2 = f2s_from_double(1.0 / (hg * hg));
      k.ih2_hi[g] = ih2.hi;
      k.ih2_lo[g] = ih2.lo;
    }
    k.inv_dt = T(1.0 / c->g.dt);
    k.half_inv_re = T(0.5 / c->g.re);
    k.inv_re = T(1.0 / c->g.re);
    k.U = T(c->g.uinf[0]);
    k.V = T(c->g.uinf[1]);
    FSI_CUDA_TRY(pdl_launch(k_rhs<T, TF>, gr, dim3(b), 0, c->stream, w_all, (const TF*)s_all, (T*)c->nprev_all,
                            (T*)c->rhs_all, c->lvl_elems, c->ps, c->nx, c->ny, k, first, delta, defect));
    prof_mark(c, KC_RHS);
  }
  FSI_CUDA_TRY(cudaGetLastError());
  // The x-transforms need only each level's own right-hand side (the coarser level's solution enters
  // through the ring terms of pass Y), so the FFT path takes all levels in one launch, each into its own
  // scratch slot; the chain of dependent launches per step is two shorter for three levels.
  const bool batch = (c->G > 1 || delta) && !use_gemm<T>(c, 0) && !use_gemm<T>(c, 1);
  if (delta && !batch) return FSI_ERR_UNSUPPORTED;  // the increment form runs on the FFT passes
  if (batch) {
    const fsi_status st = xf_pass<T>(c, (const T*)c->rhs_all, delta ? 2 * c->G : c->G);
    if (st != FSI_OK) return st;
  }
  for (int g = c->G - 1; g >= 0; --g) {
    const int ring = g < c->G - 1;
    const int inc = delta;
    if (ring) {
      fsi_status st = ring_spectra_t<T, TF>(c, g, inc);
      if (st != FSI_OK) return st;
    }
    TF* wg = w_all + (long)g * c->lvl_elems;
    TF* sg = s_all + (long)g * c->lvl_elems;
    fsi_status st;
    if (batch) {
      st = y_pass<T>(c, g, (const T*)c->T1 + (long)g * c->Nx * c->ldT, ring,
                     inc ? (const T*)c->T1 + (long)(c->G + g) * c->Nx * c->ldT : nullptr);
      if (st == FSI_OK) st = xi_pass<T, TF>(c, wg, sg, inc ? 2 : 0);
    } else {
      st = level_solve_t<T, TF>(c, g, (const T*)c->rhs_all + (long)g * c->lvl_elems, wg, sg, ring, inc ? 2 : 0);
    }
    if (st != FSI_OK) return st;
  }
  return FSI_OK;
}

template <typename T, typename TF = T>
fsi_status corrector_t(fsi_ctx* c) {
  const int wi = c->ni + 6, wj = c->nj + 6;
  dim3 gr((wi + 31) / 32, (wj + 3) / 4);
  const double scale = c->ds / (c->g.h * c->g.h);
  prof_mark(c, KC_SRC);
  // the curl of the spread stress in double whenever the fields carry more than float precision
  using TS = typename std::conditional<std::is_same<TF, f2s>::value, double, TF>::type;
  FSI_CUDA_TRY(pdl_launch(k_src<T, TS>, gr, dim3(128), 0, c->stream, (T*)c->src, c->ps, c->nx, c->ny, c->d_pidx, c->d_pcij, c->d_pw, c->d_f, c->nb, c->ni,
                                      c->i_lo, c->i_hi, c->j_lo, c->j_hi, c->d_ctrl + 8, TS(scale / c->g.h), c->n_box));
  prof_mark(c, KC_SRC);
  c->launches_per_step += 1;
  FSI_CUDA_TRY(cudaGetLastError());
  const fsi_status st = launch_appended_source(c);  // E^T f of the appended points (appended.cu)
  if (st != FSI_OK) return st;
  return level_solve_t<T, TF>(c, 0, (const T*)c->src, (TF*)c->w_all, (TF*)c->s_all, 0, 1);
}

}  // namespace

// One level solve whose right-hand side and fields are all in the transform precision of the context (scratch
// fields of the offline stage and the operator tests; not the double level fields of the mixed mode).
fsi_status launch_level_solve(fsi_ctx* c, int g, const void* rhs, void* w, void* s, int use_ring, int mode) {
  if (c->prec == FSI_PREC_FP64) return level_solve_t<double>(c, g, (const double*)rhs, (double*)w, (double*)s, use_ring, mode);
  return level_solve_t<float>(c, g, (const float*)rhs, (float*)w, (float*)s, use_ring, mode);
}

fsi_status launch_predictor(fsi_ctx* c, int first) {
  if (c->prec == FSI_PREC_FP64) return predictor_t<double>(c, first);
  if (c->prec == FSI_PREC_MIXED) return predictor_t<float, f2s>(c, first);
  return predictor_t<float>(c, first);
}

fsi_status launch_corrector(fsi_ctx* c) {
  if (c->prec == FSI_PREC_FP64) return corrector_t<double>(c);
  if (c->prec == FSI_PREC_MIXED) return corrector_t<float, f2s>(c);
  return corrector_t<float>(c);
}
