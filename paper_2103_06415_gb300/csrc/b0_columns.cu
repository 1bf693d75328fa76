// Offline stage exactly as Algorithm 1 states it: column u of B0 is the action
//   B0 e_u = E0 C (C^T A C)^{-1} C^T E0^T e_u                                   (Eq. action)
// i.e. one DST-diagonalised solve (Lap^{-1} A_w^{-1}, finest level, zero boundary values) per unknown.
// Columns are processed in batches (columns of several Omega_0 boxes on one grid may share a batch): the source C^T E0^T e_u is a 6-vertex stencil (the transpose of the
// E0 C row stencil), the three DST passes run with the batch on gridDim.y, and E0 C is applied at every
// Omega_0 point of each solved streamfunction.  B0 is symmetric, so column u is stored as row u (coalesced).
// The arithmetic precision of the solves is the context's (float or double); B0 is stored in double.
#include <chrono>
#include <vector>
#include "spec.cuh"

namespace {

// src[c] (interior layout, row stride ps, batch stride lvl) <- C^T E0^T e_u for the global unknown
// u = col0 + c of the concatenated boxes; the batch buffer is zeroed before this kernel.
template <typename T>
__global__ void k_col_source(T* __restrict__ src, long lvl, long ps, long col0, int ncols,
                             const B0Box* __restrict__ bx, int n_boxes, double inv2h) {
  const int c = blockIdx.x * blockDim.y + threadIdx.y, t = threadIdx.x;  // t < 6
  if (c >= ncols || t >= 6) return;
  const long ug = col0 + c;
  const B0Box b = bx[b0_find_box(bx, n_boxes, ug)];
  const int u = (int)(ug - b.row_off), comp = u / b.n_sd, p = u - comp * b.n_sd;
  const int I = b.i_lo + p % b.ni, J = b.j_lo + p / b.ni;
  int dx, dy;
  double w;
  e0c_stencil(comp, t, inv2h, &dx, &dy, &w);
  src[(long)c * lvl + (long)(J + dy - 1) * ps + (I + dx - 1)] = T(w);
}

// row u of its box's B0 <- E0 C s_c at every Omega_0 unknown r of that box (stencil applied to the solved
// field); blockIdx.y is the column of the batch
template <typename T>
__global__ void k_col_gather(double* __restrict__ out, const T* __restrict__ s, long lvl, long ps, long col0,
                             int ncols, const B0Box* __restrict__ bx, int n_boxes, double inv2h) {
  const int c = blockIdx.y;
  if (c >= ncols) return;
  const long ug = col0 + c;
  const B0Box b = bx[b0_find_box(bx, n_boxes, ug)];
  const long n2 = 2L * b.n_sd;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n2) return;
  const int comp = r / b.n_sd, p = r - comp * b.n_sd;
  const int I = b.i_lo + p % b.ni, J = b.j_lo + p / b.ni;
  const T* sc = s + (long)c * lvl;
  double acc = 0.0;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    int dx, dy;
    double w;
    e0c_stencil(comp, t, inv2h, &dx, &dy, &w);
    acc += w * (double)sc[(long)(J + dy) * ps + (I + dx)];
  }
  out[b.out_off + (ug - b.row_off) * n2 + r] = acc;
}

template <typename T>
void set_attrs() {
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
  cudaFuncSetAttribute(dst::k_xf<T, 1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_ysolve<T, 1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(dst::k_xi<T, 1, T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

// Launch shape of the passes for a length r3 2^logP (as the fluid step's): 4 PER threads = nf 2^logP.
struct Shape {
  int nthr, per, nf, r3, logP, L;
};
Shape shape_for(int logP, int r3) {
  const int P = 1 << logP;
  Shape c;
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

#define COL_DISPATCH(cfg, LAUNCH)   \
  do {                              \
    if ((cfg).r3 == 3)              \
      LAUNCH(1, 3);                 \
    else if ((cfg).per == 1)        \
      LAUNCH(1, 1);                 \
    else if ((cfg).per == 2)        \
      LAUNCH(2, 1);                 \
    else                            \
      LAUNCH(4, 1);                 \
  } while (0)

template <typename T>
fsi_status columns_t(fsi_ctx* c, std::vector<B0Box>& boxes, double* out) {
  using c2 = typename C2<T>::t;
  const int Nx = c->Nx, Ny = c->Ny;
  const long lvl = c->lvl_elems, ps = c->ps;
  const long t1 = (long)Nx * c->ldT, t2 = (long)Ny * c->ldX;
  b0_layout(boxes);
  const int n_boxes = (int)boxes.size();
  long n2 = 0, max_n2 = 0;  // all columns of all boxes; longest column
  for (const B0Box& b : boxes) {
    n2 += 2L * b.n_sd;
    if (2L * b.n_sd > max_n2) max_n2 = 2L * b.n_sd;
  }
  const size_t per_col = ((size_t)3 * lvl + t1 + 2 * t2) * sizeof(T);
  size_t Bz = ((size_t)2 << 30) / per_col;  // batch of columns in ~2 GiB of scratch
  if (Bz > 256) Bz = 256;
  if (Bz < 1) Bz = 1;
  const int B = (int)Bz;
  set_attrs<T>();
  T *src = nullptr, *T1 = nullptr, *T2w = nullptr, *T2s = nullptr, *fw = nullptr, *fs = nullptr;
  B0Box* d_bx = nullptr;
  fsi_status st = FSI_OK;
  if (ctx_dev_malloc(c, (void**)&d_bx, (size_t)n_boxes * sizeof(B0Box)) != cudaSuccess || ctx_dev_malloc(c, (void**)&src, (size_t)B * lvl * sizeof(T)) != cudaSuccess ||
      ctx_dev_malloc(c, (void**)&T1, (size_t)B * t1 * sizeof(T)) != cudaSuccess ||
      ctx_dev_malloc(c, (void**)&T2w, (size_t)B * t2 * sizeof(T)) != cudaSuccess ||
      ctx_dev_malloc(c, (void**)&T2s, (size_t)B * t2 * sizeof(T)) != cudaSuccess ||
      ctx_dev_malloc(c, (void**)&fw, (size_t)B * lvl * sizeof(T)) != cudaSuccess ||
      ctx_dev_malloc(c, (void**)&fs, (size_t)B * lvl * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    st = FSI_ERR_OOM;
  } else if (cudaMemcpyAsync(d_bx, boxes.data(), (size_t)n_boxes * sizeof(B0Box), cudaMemcpyHostToDevice,
                             c->stream) != cudaSuccess) {
    st = FSI_ERR_CUDA;
  }
  const Shape cx = shape_for(c->logPx, c->r3x), cy = shape_for(c->logPy, c->r3y);
  const int Lx = cx.L, Ly = cy.L;
  const c2* twx = (const c2*)c->twx;
  const c2* twy = (const c2*)c->twy;
  const double h = c->g.h, inv2h = 0.5 / h;
  const dst::SpecParams<T> sp = spec_params<T>(c, h, nullptr);
  for (long col0 = 0; st == FSI_OK && col0 < n2; col0 += B) {
    const int nc = n2 - col0 < B ? (int)(n2 - col0) : B;
    if (cudaMemsetAsync(src, 0, (size_t)nc * lvl * sizeof(T), c->stream) != cudaSuccess) {
      st = FSI_ERR_CUDA;
      break;
    }
    k_col_source<T><<<(nc + 31) / 32, dim3(8, 32), 0, c->stream>>>(src, lvl, ps, col0, nc, d_bx, n_boxes, inv2h);
    {
      dim3 grid((Ny + 2 * cx.nf - 1) / (2 * cx.nf), nc);
      const size_t sm = dst::pass_smem<T>((size_t)cx.nf * Lx, Lx);
#define XF(P, R) dst::k_xf<T, P, R><<<grid, cx.nthr, sm, c->stream>>>(src, ps, lvl, Ny, Nx, T1, c->ldT, t1, twx, cx.logP, cx.nf)
      COL_DISPATCH(cx, XF);
#undef XF
    }
    {
      dim3 grid((Nx + 2 * cy.nf - 1) / (2 * cy.nf), nc);
      const size_t sm = dst::pass_smem<T>((size_t)2 * cy.nf * Ly, Ly);
#define YS(P, R) dst::k_ysolve<T, P, R><<<grid, cy.nthr, sm, c->stream>>>(T1, c->ldT, t1, Nx, Ny, T2w, T2s, c->ldX, t2, twy, cy.logP, cy.nf, sp, (const T*)nullptr)
      COL_DISPATCH(cy, YS);
#undef YS
    }
    {
      dim3 grid(dst::xi_blocks(Ny, cx.nf), nc);
      const size_t sm = dst::pass_smem<T>((size_t)cx.nf * Lx, Lx);
#define XI(P, R) dst::k_xi<T, P, T, R><<<grid, cx.nthr, sm, c->stream>>>(T2w, T2s, c->ldX, t2, Ny, Nx, fw, fs, ps, lvl, 0, twx, cx.logP, cx.nf)
      COL_DISPATCH(cx, XI);
#undef XI
    }
    k_col_gather<T><<<dim3((unsigned)((max_n2 + 255) / 256), nc), 256, 0, c->stream>>>(out, fs, lvl, ps, col0, nc,
                                                                                       d_bx, n_boxes, inv2h);
    if (cudaGetLastError() != cudaSuccess) st = FSI_ERR_CUDA;
  }
  if (st == FSI_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = FSI_ERR_CUDA;
  ctx_dev_free(c, src);
  ctx_dev_free(c, T1);
  ctx_dev_free(c, T2w);
  ctx_dev_free(c, T2s);
  ctx_dev_free(c, fw);
  ctx_dev_free(c, fs);
  ctx_dev_free(c, d_bx);
  return st;
}

}  // namespace

fsi_status b0_columns(fsi_ctx* c, std::vector<B0Box>& boxes, double* out) {
  return c->prec == FSI_PREC_FP64 ? columns_t<double>(c, boxes, out) : columns_t<float>(c, boxes, out);
}

fsi_status build_b0_columns(fsi_ctx* c) {
  auto t0 = std::chrono::steady_clock::now();
  std::vector<B0Box> one(1, ctx_box(c));
  const fsi_status st = b0_columns(c, one, c->B0);
  c->b0_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st;
}
