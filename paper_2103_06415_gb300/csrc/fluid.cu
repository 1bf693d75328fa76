// Fluid part of one time step on the nested levels: advection + right-hand side (App. A, AB2/CN),
// multidomain coupling (Sec. 5, far-field multidomain), the DST-diagonalised predictor solves
// (Eq. predictor2) and the corrector (Eq. corrector2) with its surface-stress source.
#include <cstdio>
#include <type_traits>
#include "dst.cuh"
#include "internal.h"

namespace {

// ---------------------------------------------------------------------------------------------
// Launch shapes of the FFT passes: elements per CTA = 4 * PER * threads = nf * L.
struct FftCfg {
  int nthr, per, nf;
};
FftCfg fft_cfg(int logL) {
  const int L = 1 << logL;
  FftCfg c;
  c.nthr = L / 4;
  if (c.nthr < 32) c.nthr = 32;
  if (c.nthr > 256) c.nthr = 256;
  c.per = 1;
  while (4 * c.per * c.nthr < L) c.per *= 2;
  c.nf = 4 * c.per * c.nthr / L;
  return c;
}

template <typename T>
void set_smem_limits() {
  static bool done = false;
  if (done) return;
  done = true;
  const int big = 200 * 1024;
  cudaFuncSetAttribute(dst::k_xf<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xf<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xf<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_ysolve<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_ysolve<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_ysolve<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xi<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xi<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xi<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_vec_dst<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_vec_dst<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_vec_dst<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

// ---------------------------------------------------------------------------------------------
// O1: coarse vorticity strictly inside a finer level <- coincident value of the finest such level.
template <typename T>
__global__ void k_inject(T* __restrict__ w_all, long lvl, long ps, int nx, int ny) {
  const int g = blockIdx.z + 1;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I < 1 || I >= nx || J < 1 || J >= ny) return;
  int gi = g, ii = I, jj = J;
  // descend while strictly inside the next finer level
  while (gi > 0 && abs(2 * ii - nx) < nx / 2 && abs(2 * jj - ny) < ny / 2) {
    ii = 2 * ii - nx / 2;
    jj = 2 * jj - ny / 2;
    --gi;
  }
  if (gi == g) return;
  w_all[(long)g * lvl + (long)J * ps + I] = w_all[(long)gi * lvl + (long)jj * ps + ii];
}

// O2: advection N = div(u w) with vertex-averaged velocities (reading R7) and
// rhs = w/dt + lap_h w/(2 Re) - 3/2 N^n + 1/2 N^{n-1}.
template <typename T>
__global__ void k_rhs(const T* __restrict__ w_all, const T* __restrict__ s_all, T* __restrict__ np_all,
                      T* __restrict__ rhs_all, long lvl, long ps, int nx, int ny, double h0, double dt, double re,
                      double U, double V, int first) {
  const int g = blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (i >= nx || j >= ny) return;
  const T* w = w_all + (long)g * lvl;
  const T* s = s_all + (long)g * lvl;
  const T h = T(h0 * (double)(1 << g));
  const T i2h = T(0.5) / h;
  const long o = (long)j * ps + i;
  const T wc = w[o], we = w[o + 1], ww = w[o - 1], wn = w[o + ps], wsx = w[o - ps];
  // ubar at (i+-1, j) = (s[j+1] - s[j-1])/(2h) + U ; vbar at (i, j+-1) = -(s[i+1] - s[i-1])/(2h) + V
  const T ue = (s[o + ps + 1] - s[o - ps + 1]) * i2h + T(U);
  const T uw = (s[o + ps - 1] - s[o - ps - 1]) * i2h + T(U);
  const T vn = -(s[o + ps + 1] - s[o + ps - 1]) * i2h + T(V);
  const T vs = -(s[o - ps + 1] - s[o - ps - 1]) * i2h + T(V);
  const T n = (ue * we - uw * ww) * i2h + (vn * wn - vs * wsx) * i2h;
  const T lap = (we + ww + wn + wsx - T(4) * wc) / (h * h);
  T* np = np_all + (long)g * lvl;
  const long oi = (long)(j - 1) * ps + (i - 1);
  const T nold = first ? n : np[o];
  np[o] = n;
  rhs_all[(long)g * lvl + oi] = wc * T(1.0 / dt) + lap * T(0.5 / re) - T(1.5) * n + T(0.5) * nold;
}

// O3 boundary of level g from level g+1 (injection at coincident vertices, midpoint average otherwise).
template <typename T>
__global__ void k_ring(T* __restrict__ wf, T* __restrict__ sf, const T* __restrict__ wc, const T* __restrict__ sc,
                       long ps, int nx, int ny) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nb = nx + 1, nside = ny - 1;
  int i, j;
  if (t < nb) {
    i = t;
    j = 0;
  } else if (t < 2 * nb) {
    i = t - nb;
    j = ny;
  } else if (t < 2 * nb + nside) {
    i = 0;
    j = t - 2 * nb + 1;
  } else if (t < 2 * nb + 2 * nside) {
    i = nx;
    j = t - 2 * nb - nside + 1;
  } else {
    return;
  }
  const int a = i + nx / 2, b = j + ny / 2;  // position in half-coarse units
  const int I0 = a >> 1, J0 = b >> 1;
  const int I1 = I0 + (a & 1), J1 = J0 + (b & 1);
  const long o00 = (long)J0 * ps + I0, o11 = (long)J1 * ps + I1;
  const T w = T(0.5) * (wc[o00] + wc[o11]);
  const T s = T(0.5) * (sc[o00] + sc[o11]);
  wf[(long)j * ps + i] = w;
  sf[(long)j * ps + i] = s;
}

// O5 source: src = (ds/h^2) curl_h(E0^T P^T f) on the level-0 vertices near the body.  Deterministic
// gather: every vertex sums over all body points with a fixed order and reduction tree (no atomics), so a
// run gives the same bits every time.  Face weights: P row (hat, 4 nodes) times the E0 stencil
// (1/6, 2/3, 1/6) x (1/2, 1/2).
__device__ __forceinline__ double wx3(int d) { return d == 0 ? 2.0 / 3.0 : ((d == 1 || d == -1) ? 1.0 / 6.0 : 0.0); }

// Contribution of body point p to the four faces around vertex (i, j) that enter the curl.
__device__ __forceinline__ void point_faces(int i, int j, int ci, int cj, const double* w, double fxp, double fyp,
                                            double* fve, double* fvw, double* fun, double* fus) {
  if (i < ci - 2 || i > ci + 4 || j < cj - 2 || j > cj + 4) return;
  double ve = 0.0, vw = 0.0, un = 0.0, us = 0.0;
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int vi = ci + a, vj = cj + b;
      const double wp = w[2 * b + a];
      // u-face (fi, fj+1/2): wx3(fi - vi) * 1/2 if fj - vj in {-1, 0}; v-face (fi+1/2, fj) likewise
      const int dn = j - vj, ds_ = j - 1 - vj;
      un += wp * wx3(i - vi) * ((dn == 0 || dn == -1) ? 0.5 : 0.0);
      us += wp * wx3(i - vi) * ((ds_ == 0 || ds_ == -1) ? 0.5 : 0.0);
      const int de = i - vi, dw = i - 1 - vi;
      ve += wp * ((de == 0 || de == -1) ? 0.5 : 0.0) * wx3(j - vj);
      vw += wp * ((dw == 0 || dw == -1) ? 0.5 : 0.0) * wx3(j - vj);
    }
  *fve += ve * fyp;
  *fvw += vw * fyp;
  *fun += un * fxp;
  *fus += us * fxp;
}

// One warp per vertex: lanes take body points p = lane, lane + 32, ... and the four face sums are reduced
// with a fixed shuffle tree.  Vertices outside the box written by the FSI kernel (ctrl[8..11]) are set to
// zero.  Grid: x covers the Omega_0 box grown by 3 cells in tiles of 32 vertices, y its rows.
template <typename T>
__global__ void __launch_bounds__(256) k_src(T* __restrict__ src, long ps, int nx, int ny, const int* __restrict__ pidx,
                                             const double* __restrict__ pw, const double* __restrict__ f, int nb, int ni,
                                             int i_lo, int i_hi, int j_lo, int j_hi, const int* __restrict__ box,
                                             double scale, double h) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int j = j_lo - 3 + blockIdx.y;
  const int i0 = i_lo - 3 + blockIdx.x * 32;
  if (j < 1 || j > ny - 1 || j > j_hi + 3) return;
  const int bi0 = box[0], bi1 = box[1], bj0 = box[2], bj1 = box[3];
  const bool row_in = j >= bj0 && j <= bj1;
  if (tid < 32) {
    const int i = i0 + tid;
    if (i >= 1 && i <= nx - 1 && i <= i_hi + 3 && !(row_in && i >= bi0 && i <= bi1))
      src[(long)(j - 1) * ps + (i - 1)] = T(0);
  }
  if (!row_in) return;
  for (int v = wid; v < 32; v += blockDim.x >> 5) {
    const int i = i0 + v;
    if (i < 1 || i > nx - 1 || i > i_hi + 3 || i < bi0 || i > bi1) continue;  // warp-uniform
    double fve = 0.0, fvw = 0.0, fun = 0.0, fus = 0.0;
    for (int p = lane; p < nb; p += 32) {
      const int n0 = pidx[4 * p];
      const double w[4] = {pw[4 * p], pw[4 * p + 1], pw[4 * p + 2], pw[4 * p + 3]};
      point_faces(i, j, n0 % ni + i_lo, n0 / ni + j_lo, w, f[p], f[nb + p], &fve, &fvw, &fun, &fus);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      fve += __shfl_xor_sync(0xffffffffu, fve, o);
      fvw += __shfl_xor_sync(0xffffffffu, fvw, o);
      fun += __shfl_xor_sync(0xffffffffu, fun, o);
      fus += __shfl_xor_sync(0xffffffffu, fus, o);
    }
    // curl at (i,j): (Fv(i+1/2,j) - Fv(i-1/2,j))/h - (Fu(i,j+1/2) - Fu(i,j-1/2))/h
    if (lane == 0) src[(long)(j - 1) * ps + (i - 1)] = T(scale * ((fve - fvw) - (fun - fus)) / h);
  }
}

// ---------------------------------------------------------------------------------------------
// Pass p of the sine transforms runs as a tensor-core GEMM (FP32 contexts that chose it; dst_gemm.cu).
template <typename T>
bool use_gemm(const fsi_ctx* c, int p) {
  return std::is_same<T, float>::value && c->gd && c->dst_gemm[p];
}

template <typename T>
fsi_status level_solve_t(fsi_ctx* c, int g, const T* rhs, T* w, T* s, int use_ring, int mode) {
  using c2 = typename C2<T>::t;
  set_smem_limits<T>();
  const FftCfg cx = fft_cfg(c->logLx), cy = fft_cfg(c->logLy);
  const int Lx = 1 << c->logLx, Ly = 1 << c->logLy;
  const c2* twx = (const c2*)c->twx;
  const c2* twy = (const c2*)c->twy;
  // XF
  prof_mark(c, KC_XF);
  if (use_gemm<T>(c, 0)) {
    const fsi_status st = gemm_xf(c, (const float*)rhs);
    if (st != FSI_OK) return st;
  } else {
    dim3 grid((c->Ny + 2 * cx.nf - 1) / (2 * cx.nf), 1);
    const size_t sm = (size_t)cx.nf * Lx * sizeof(c2);
    switch (cx.per) {
      case 1: dst::k_xf<T, 1><<<grid, cx.nthr, sm, c->stream>>>(rhs, c->ps, 0, c->Ny, c->Nx, (T*)c->T1, c->ldT, 0, twx, c->logLx, cx.nf); break;
      case 2: dst::k_xf<T, 2><<<grid, cx.nthr, sm, c->stream>>>(rhs, c->ps, 0, c->Ny, c->Nx, (T*)c->T1, c->ldT, 0, twx, c->logLx, cx.nf); break;
      default: dst::k_xf<T, 4><<<grid, cx.nthr, sm, c->stream>>>(rhs, c->ps, 0, c->Ny, c->Nx, (T*)c->T1, c->ldT, 0, twx, c->logLx, cx.nf); break;
    }
  }
  prof_mark(c, KC_XF);
  // Y
  prof_mark(c, KC_YSOLVE);
  {
    dst::SpecParams<T> sp;
    sp.lx = c->lx;
    sp.ly = c->ly;
    sp.sx1 = c->sx1;
    sp.sxN = c->sxN;
    sp.sy1 = c->sy1;
    sp.syN = c->syN;
    sp.ring = use_ring ? (const T*)c->ring : nullptr;
    sp.ring_ld = c->ring_ld;
    const double h = c->g.h * (double)(1 << g);
    sp.inv_h2 = 1.0 / (h * h);
    sp.inv_dt = 1.0 / c->g.dt;
    sp.inv_2re = 0.5 / c->g.re;
    sp.norm = 4.0 / ((double)c->Mx * (double)c->My);
    sp.Mx = c->Mx;
    sp.My = c->My;
    if (use_gemm<T>(c, 1)) {
      if constexpr (std::is_same<T, float>::value) {
        const fsi_status st = gemm_ysolve(c, sp);
        if (st != FSI_OK) return st;
      }
    } else {
      dim3 grid((c->Nx + 2 * cy.nf - 1) / (2 * cy.nf), 1);
      const size_t sm = (size_t)3 * cy.nf * Ly * sizeof(c2);
      switch (cy.per) {
        case 1: dst::k_ysolve<T, 1><<<grid, cy.nthr, sm, c->stream>>>((const T*)c->T1, c->ldT, 0, c->Nx, c->Ny, (T*)c->T2w, (T*)c->T2s, c->ldX, 0, twy, c->logLy, cy.nf, sp); break;
        case 2: dst::k_ysolve<T, 2><<<grid, cy.nthr, sm, c->stream>>>((const T*)c->T1, c->ldT, 0, c->Nx, c->Ny, (T*)c->T2w, (T*)c->T2s, c->ldX, 0, twy, c->logLy, cy.nf, sp); break;
        default: dst::k_ysolve<T, 4><<<grid, cy.nthr, sm, c->stream>>>((const T*)c->T1, c->ldT, 0, c->Nx, c->Ny, (T*)c->T2w, (T*)c->T2s, c->ldX, 0, twy, c->logLy, cy.nf, sp); break;
      }
    }
  }
  prof_mark(c, KC_YSOLVE);
  // XI: 2*nf rows per CTA; rows j, j+1 of w share one FFT, rows j, j+1 of s another
  prof_mark(c, KC_XI);
  if (use_gemm<T>(c, 2)) {
    const fsi_status st = gemm_xi(c, (float*)w, (float*)s, mode);
    if (st != FSI_OK) return st;
  } else {
    dim3 grid((c->Ny + 2 * cx.nf - 1) / (2 * cx.nf), 1);
    const size_t sm = (size_t)2 * cx.nf * Lx * sizeof(c2);
    switch (cx.per) {
      case 1: dst::k_xi<T, 1><<<grid, cx.nthr, sm, c->stream>>>((const T*)c->T2w, (const T*)c->T2s, c->ldX, 0, c->Ny, c->Nx, w, s, c->ps, 0, mode, twx, c->logLx, cx.nf); break;
      case 2: dst::k_xi<T, 2><<<grid, cx.nthr, sm, c->stream>>>((const T*)c->T2w, (const T*)c->T2s, c->ldX, 0, c->Ny, c->Nx, w, s, c->ps, 0, mode, twx, c->logLx, cx.nf); break;
      default: dst::k_xi<T, 4><<<grid, cx.nthr, sm, c->stream>>>((const T*)c->T2w, (const T*)c->T2s, c->ldX, 0, c->Ny, c->Nx, w, s, c->ps, 0, mode, twx, c->logLx, cx.nf); break;
    }
  }
  prof_mark(c, KC_XI);
  FSI_CUDA_TRY(cudaGetLastError());
  c->launches_per_step += 3;
  return FSI_OK;
}

template <typename T>
fsi_status ring_spectra_t(fsi_ctx* c, int g) {
  using c2 = typename C2<T>::t;
  T* wf = (T*)c->w_all + (long)g * c->lvl_elems;
  T* sf = (T*)c->s_all + (long)g * c->lvl_elems;
  const T* wc = (const T*)c->w_all + (long)(g + 1) * c->lvl_elems;
  const T* sc = (const T*)c->s_all + (long)(g + 1) * c->lvl_elems;
  const int nring = 2 * (c->nx + 1) + 2 * (c->ny - 1);
  prof_mark(c, KC_RING);
  k_ring<T><<<(nring + 127) / 128, 128, 0, c->stream>>>(wf, sf, wc, sc, c->ps, c->nx, c->ny);
  prof_mark(c, KC_RING);
  c->launches_per_step += 3;
  // four vectors of length Ny (wL, wR, sL, sR) and four of length Nx (wB, wT, sB, sT)
  for (int side = 0; side < 2; ++side) {
    const int logL = side == 0 ? c->logLy : c->logLx;
    const int N = side == 0 ? c->Ny : c->Nx;
    const int L = 1 << logL;
    const int nthr = L / 4 < 256 ? L / 4 : 256;
    const int per = L / (4 * nthr);
    const size_t sm = (size_t)(1 << logL) * sizeof(c2);
    const T* const* srcs = (const T* const*)(c->ring_src + (long)g * 8 + side * 4);
    const long* es = c->ring_es + (long)g * 8 + side * 4;
    T* const* dsts = (T* const*)(c->ring_dst + (long)g * 8 + side * 4);
    const c2* tw = (const c2*)(side == 0 ? c->twy : c->twx);
    prof_mark(c, KC_VECDST);
    switch (per) {
      case 1: dst::k_vec_dst<T, 1><<<2, nthr, sm, c->stream>>>(srcs, es, 4, N, dsts, tw, logL); break;
      case 2: dst::k_vec_dst<T, 2><<<2, nthr, sm, c->stream>>>(srcs, es, 4, N, dsts, tw, logL); break;
      default: dst::k_vec_dst<T, 4><<<2, nthr, sm, c->stream>>>(srcs, es, 4, N, dsts, tw, logL); break;
    }
    prof_mark(c, KC_VECDST);
  }
  FSI_CUDA_TRY(cudaGetLastError());
  return FSI_OK;
}

template <typename T>
fsi_status predictor_t(fsi_ctx* c, int first) {
  T* w_all = (T*)c->w_all;
  T* s_all = (T*)c->s_all;
  if (c->G > 1) {
    dim3 b(32, 8), gr((c->nx + 31) / 32, (c->ny + 7) / 8, c->G - 1);
    prof_mark(c, KC_INJECT);
    k_inject<T><<<gr, b, 0, c->stream>>>(w_all, c->lvl_elems, c->ps, c->nx, c->ny);
    prof_mark(c, KC_INJECT);
    c->launches_per_step += 1;
  }
  {
    dim3 b(32, 8), gr((c->Nx + 31) / 32, (c->Ny + 7) / 8, c->G);
    c->launches_per_step += 1;
    prof_mark(c, KC_RHS);
    k_rhs<T><<<gr, b, 0, c->stream>>>(w_all, s_all, (T*)c->nprev_all, (T*)c->rhs_all, c->lvl_elems, c->ps, c->nx,
                                      c->ny, c->g.h, c->g.dt, c->g.re, c->g.uinf[0], c->g.uinf[1], first);
    prof_mark(c, KC_RHS);
  }
  FSI_CUDA_TRY(cudaGetLastError());
  for (int g = c->G - 1; g >= 0; --g) {
    const int ring = g < c->G - 1;
    if (ring) {
      fsi_status st = ring_spectra_t<T>(c, g);
      if (st != FSI_OK) return st;
    }
    fsi_status st = level_solve_t<T>(c, g, (const T*)c->rhs_all + (long)g * c->lvl_elems,
                                     w_all + (long)g * c->lvl_elems, s_all + (long)g * c->lvl_elems, ring, 0);
    if (st != FSI_OK) return st;
  }
  return FSI_OK;
}

template <typename T>
fsi_status corrector_t(fsi_ctx* c) {
  dim3 b(32, 8);
  const int wi = c->ni + 6, wj = c->nj + 6;
  dim3 gr((wi + 31) / 32, wj);
  const double scale = c->ds / (c->g.h * c->g.h);
  prof_mark(c, KC_SRC);
  k_src<T><<<gr, 256, 0, c->stream>>>((T*)c->src, c->ps, c->nx, c->ny, c->d_pidx, c->d_pw, c->d_f, c->nb, c->ni,
                                      c->i_lo, c->i_hi, c->j_lo, c->j_hi, c->d_ctrl + 8, scale, c->g.h);
  prof_mark(c, KC_SRC);
  c->launches_per_step += 1;
  FSI_CUDA_TRY(cudaGetLastError());
  return level_solve_t<T>(c, 0, (const T*)c->src, (T*)c->w_all, (T*)c->s_all, 0, 1);
}

}  // namespace

fsi_status launch_level_solve(fsi_ctx* c, int g, const void* rhs, void* w, void* s, int use_ring, int mode) {
  if (c->prec == FSI_PREC_FP64) return level_solve_t<double>(c, g, (const double*)rhs, (double*)w, (double*)s, use_ring, mode);
  return level_solve_t<float>(c, g, (const float*)rhs, (float*)w, (float*)s, use_ring, mode);
}

fsi_status launch_predictor(fsi_ctx* c, int first) {
  if (c->prec == FSI_PREC_FP64) return predictor_t<double>(c, first);
  return predictor_t<float>(c, first);
}

fsi_status launch_corrector(fsi_ctx* c) {
  if (c->prec == FSI_PREC_FP64) return corrector_t<double>(c);
  return corrector_t<float>(c);
}
