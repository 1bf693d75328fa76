// Appended sub-domain points (Sec. 3.1.1): the exact points of stationary bodies join Omega_0 with weight one
// and are interpolated with E itself.  The operator gains their rows and columns,
//   B0[a][b] = E_a C (C^T A C)^-1 C^T E_b^T      (E_x = E0 at a box vertex, E at an appended point),
// the box block comes from the chosen B0 method and is expanded into the layout in which each component's
// appended unknowns follow its n_box box unknowns; each appended column is one finest-level solve with
// homogeneous boundary values (Eq. action, Algorithm 1) in the context's precision.  B0 is symmetric: the
// solve for appended column u gives row u, and the box rows of column u by symmetry.
// In the step, P maps an appended body point to its own unknown with weight one; the right-hand side uses
// E (C s* + q_inf) at the point (fsi.cu) and the corrector spreads its stress with E^T (below).
#include <cmath>
#include <vector>
#include "internal.h"

namespace {

// face windows of the appended points (one thread per point); points closer than 2 cells to the grid
// boundary are clamped and flagged
__global__ void k_app_windows(const double* __restrict__ pts, int n, double x0, double y0, double h, int nx, int ny,
                              FaceWindow* __restrict__ out, int* bad) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  double X = (pts[2 * a] - x0) / h, Y = (pts[2 * a + 1] - y0) / h;
  if (!(X >= 2.0 && X <= nx - 2.0 && Y >= 2.0 && Y <= ny - 2.0)) {
    atomicExch(bad, 1);
    X = fmin(fmax(isfinite(X) ? X : 2.0, 2.0), nx - 2.0);
    Y = fmin(fmax(isfinite(Y) ? Y : 2.0, 2.0), ny - 2.0);
  }
  FaceWindow f;
  f.iu = (int)floor(X) - 1;
  f.ju = (int)floor(Y - 0.5) - 1;
  f.iv = (int)floor(X - 0.5) - 1;
  f.jv = (int)floor(Y) - 1;
  for (int k = 0; k < 4; ++k) {
    f.w[k] = delta3_rn(__dsub_rn((double)(f.iu + k), X));
    f.w[4 + k] = delta3_rn(__dsub_rn(__dadd_rn((double)(f.ju + k), 0.5), Y));
    f.w[8 + k] = delta3_rn(__dsub_rn(__dadd_rn((double)(f.iv + k), 0.5), X));
    f.w[12 + k] = delta3_rn(__dsub_rn((double)(f.jv + k), Y));
  }
  out[a] = f;
}

// box operator [2 n_box]^2 into the full layout [2 n_sd]^2 (box unknown r -> r, or r + n_app for y)
__global__ void k_expand(double* __restrict__ full, const double* __restrict__ box, long n_box, long n_sd) {
  const long nb2 = 2 * n_box, n_app = n_sd - n_box;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nb2 * nb2; e += (long)gridDim.x * blockDim.x) {
    const long r = e / nb2, c = e - r * nb2;
    const long fr = r < n_box ? r : r + n_app, fc = c < n_box ? c : c + n_app;
    full[fr * 2 * n_sd + fc] = box[e];
  }
}

// source of appended column (comp, a): curl of E^T e at point a, i.e. (Fv(i+1/2,j) - Fv(i-1/2,j)) / h -
// (Fu(i,j+1/2) - Fu(i,j-1/2)) / h with the unit force's face values F; the buffer is zeroed before
template <typename T>
__global__ void k_app_col_source(T* __restrict__ src, long ps, int nx, int ny, const FaceWindow* __restrict__ win,
                                 int a, int comp, double h) {
  const FaceWindow f = win[a];
  const int t = threadIdx.x;  // 36 vertices of the 6 x 6 region from (min(iu, iv), min(ju, jv))
  if (t >= 36) return;
  const int i = min(f.iu, f.iv) + t % 6, j = min(f.ju, f.jv) + t / 6;
  if (i < 1 || i > nx - 1 || j < 1 || j > ny - 1) return;  // boundary vertices carry no unknown
  double val = 0.0;
  if (comp == 0) {  // -(Fu(i, j) - Fu(i, j - 1)) / h, Fu on u face (i, j) = w[i - iu] w[4 + j - ju]
    const int d = i - f.iu, en = j - f.ju, es = j - 1 - f.ju;
    double fn = 0.0, fs = 0.0;
    if (d >= 0 && d < 4 && en >= 0 && en < 4) fn = f.w[d] * f.w[4 + en];
    if (d >= 0 && d < 4 && es >= 0 && es < 4) fs = f.w[d] * f.w[4 + es];
    val = -(fn - fs) / h;
  } else {  // (Fv(i, j) - Fv(i - 1, j)) / h, Fv on v face (i, j) = w[8 + i - iv] w[12 + j - jv]
    const int e = j - f.jv, de = i - f.iv, dw = i - 1 - f.iv;
    double fe = 0.0, fw = 0.0;
    if (e >= 0 && e < 4 && de >= 0 && de < 4) fe = f.w[8 + de] * f.w[12 + e];
    if (e >= 0 && e < 4 && dw >= 0 && dw < 4) fw = f.w[8 + dw] * f.w[12 + e];
    val = (fe - fw) / h;
  }
  src[(long)(j - 1) * ps + (i - 1)] = T(val);
}

// E_r C s at unknown r for every r (E0 C stencil at box vertices, E C at appended points) into row col of B0,
// and into column col for the box rows
template <typename T>
__global__ void k_app_col_gather(double* __restrict__ b0, long n_sd, int n_box, int ni, int i_lo, int j_lo,
                                 const T* __restrict__ s, long ps, const FaceWindow* __restrict__ win, long col,
                                 double h) {
  const long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= 2 * n_sd) return;
  const int comp = (int)(r / n_sd), p = (int)(r - comp * n_sd);
  double acc = 0.0;
  if (p < n_box) {
    const int I = i_lo + p % ni, J = j_lo + p / ni;
    const double inv2h = 0.5 / h;
    for (int t = 0; t < 6; ++t) {
      int dx, dy;
      double w;
      e0c_stencil(comp, t, inv2h, &dx, &dy, &w);
      acc += w * (double)s[(long)(J + dy) * ps + (I + dx)];
    }
  } else {
    const FaceWindow f = win[p - n_box];
    for (int e = 0; e < 4; ++e)
      for (int d = 0; d < 4; ++d) {
        if (comp == 0) {
          const long I = f.iu + d, J = f.ju + e;
          acc += (f.w[d] * f.w[4 + e]) * (((double)s[(J + 1) * ps + I] - (double)s[J * ps + I]) / h);
        } else {
          const long I = f.iv + d, J = f.jv + e;
          acc += (f.w[8 + d] * f.w[12 + e]) * (-((double)s[J * ps + I + 1] - (double)s[J * ps + I]) / h);
        }
      }
  }
  b0[col * 2 * n_sd + r] = acc;
  if (p < n_box) b0[r * 2 * n_sd + col] = acc;
}

// corrector source of the appended points' stress: (ds/h^2) curl of E^T f on the vertex box of their
// windows; inside the box that the sub-domain source kernel writes every step the value is added, outside
// it is stored (the region outside both is never written and stays zero)
template <typename T>
__global__ void k_app_src(T* __restrict__ src, long ps, int ai0, int aj0, int ai1, int aj1, int si0, int sj0, int si1,
                          int sj1, const FaceWindow* __restrict__ win, const int* __restrict__ app_pt,
                          const double* __restrict__ f, int nb, int n_app, double pre_h) {
  const int i = ai0 + (int)(blockIdx.x * blockDim.x + threadIdx.x), j = aj0 + (int)blockIdx.y;
  if (i > ai1 || j > aj1) return;
  double fun = 0.0, fus = 0.0, fve = 0.0, fvw = 0.0;
  for (int a = 0; a < n_app; ++a) {
    const FaceWindow w = win[a];
    const int p = app_pt[a];
    const int du = i - w.iu;
    if (du >= 0 && du < 4) {
      const int en = j - w.ju, es = j - 1 - w.ju;
      if (en >= 0 && en < 4) fun += (w.w[du] * w.w[4 + en]) * f[p];
      if (es >= 0 && es < 4) fus += (w.w[du] * w.w[4 + es]) * f[p];
    }
    const int ev = j - w.jv;
    if (ev >= 0 && ev < 4) {
      const int de = i - w.iv, dw = i - 1 - w.iv;
      if (de >= 0 && de < 4) fve += (w.w[8 + de] * w.w[12 + ev]) * f[nb + p];
      if (dw >= 0 && dw < 4) fvw += (w.w[8 + dw] * w.w[12 + ev]) * f[nb + p];
    }
  }
  const double v = pre_h * ((fve - fvw) - (fun - fus));
  T* o = src + (long)(j - 1) * ps + (i - 1);
  const bool inside = i >= si0 && i <= si1 && j >= sj0 && j <= sj1;
  *o = inside ? T((double)*o + v) : T(v);
}

template <typename T>
fsi_status app_columns_t(fsi_ctx* c) {
  const long lvl = c->lvl_elems;
  void *tw = nullptr, *ts = nullptr;
  if (ctx_dev_malloc(c, (void**)&tw, lvl * c->esz) != cudaSuccess || ctx_dev_malloc(c, (void**)&ts, lvl * c->esz) != cudaSuccess) {
    cudaGetLastError();
    ctx_dev_free(c, tw);
    return FSI_ERR_OOM;
  }
  fsi_status st = FSI_OK;
  if (cudaMemsetAsync(tw, 0, lvl * c->esz, c->stream) != cudaSuccess ||
      cudaMemsetAsync(ts, 0, lvl * c->esz, c->stream) != cudaSuccess)
    st = FSI_ERR_CUDA;
  for (int comp = 0; comp < 2 && st == FSI_OK; ++comp)
    for (int a = 0; a < c->n_app && st == FSI_OK; ++a) {
      if (cudaMemsetAsync(c->src, 0, lvl * c->esz, c->stream) != cudaSuccess) {
        st = FSI_ERR_CUDA;
        break;
      }
      k_app_col_source<T><<<1, 64, 0, c->stream>>>((T*)c->src, c->ps, c->nx, c->ny, c->d_app_win, a, comp, c->g.h);
      if (cudaGetLastError() != cudaSuccess) {
        st = FSI_ERR_CUDA;
        break;
      }
      st = launch_level_solve(c, 0, c->src, tw, ts, 0, 0);
      if (st != FSI_OK) break;
      const long col = (long)comp * c->n_sd + c->n_box + a;
      k_app_col_gather<T><<<(unsigned)((2 * c->n_sd + 255) / 256), 256, 0, c->stream>>>(
          c->B0, c->n_sd, c->n_box, c->ni, c->i_lo, c->j_lo, (const T*)ts, c->ps, c->d_app_win, col, c->g.h);
      if (cudaGetLastError() != cudaSuccess) st = FSI_ERR_CUDA;
    }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess && st == FSI_OK) st = FSI_ERR_CUDA;
  if (cudaMemsetAsync(c->src, 0, lvl * c->esz, c->stream) != cudaSuccess && st == FSI_OK) st = FSI_ERR_CUDA;
  cudaStreamSynchronize(c->stream);
  ctx_dev_free(c, tw);
  ctx_dev_free(c, ts);
  return st;
}

}  // namespace

fsi_status setup_appended(fsi_ctx* c) {
  if (c->n_app == 0) return FSI_OK;
  double* d_pts = nullptr;
  int* d_bad = nullptr;
  if (!(c->d_app_win = (FaceWindow*)ctx_alloc(c, (size_t)c->n_app * sizeof(FaceWindow)))) return FSI_ERR_OOM;
  if (ctx_dev_malloc(c, (void**)&d_pts, c->app_pts.size() * 8) != cudaSuccess || ctx_dev_malloc(c, (void**)&d_bad, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    ctx_dev_free(c, d_pts);
    return FSI_ERR_OOM;
  }
  int bad = 0;
  fsi_status st = FSI_OK;
  if (cudaMemcpyAsync(d_pts, c->app_pts.data(), c->app_pts.size() * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream) != cudaSuccess) {
    st = FSI_ERR_CUDA;
  } else {
    k_app_windows<<<(c->n_app + 127) / 128, 128, 0, c->stream>>>(d_pts, c->n_app, c->g.x0, c->g.y0, c->g.h, c->nx, c->ny,
                                                                c->d_app_win, d_bad);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      st = FSI_ERR_CUDA;
  }
  ctx_dev_free(c, d_pts);
  ctx_dev_free(c, d_bad);
  if (st != FSI_OK) return st;
  if (bad) {
    fsi_set_last_message("appended body point closer than 2 cells to the grid boundary");
    return FSI_ERR_BODY_OUTSIDE_SUBDOMAIN;
  }
  // vertex box of the corrector source: the windows reach 1 cell before and 4 after the window origins
  int i0 = 1 << 30, i1 = -1, j0 = 1 << 30, j1 = -1;
  const double h = c->g.h;
  for (int a = 0; a < c->n_app; ++a) {
    const double X = (c->app_pts[2 * a] - c->g.x0) / h, Y = (c->app_pts[2 * a + 1] - c->g.y0) / h;
    const int fx = (int)std::floor(X), fy = (int)std::floor(Y);
    i0 = std::min(i0, fx - 2);
    i1 = std::max(i1, fx + 3);
    j0 = std::min(j0, fy - 2);
    j1 = std::max(j1, fy + 3);
  }
  c->app_box[0] = std::max(i0, 1);
  c->app_box[1] = std::max(j0, 1);
  c->app_box[2] = std::min(i1, c->nx - 1);
  c->app_box[3] = std::min(j1, c->ny - 1);
  return FSI_OK;
}

fsi_status build_appended_b0(fsi_ctx* c) {
  // the box block by the chosen method into a temporary, expanded into c->B0
  double* full = c->B0;
  double* box = nullptr;
  const size_t nb2 = 2 * (size_t)c->n_box;
  if (ctx_dev_malloc(c, (void**)&box, nb2 * nb2 * 8) != cudaSuccess) {
    cudaGetLastError();
    return FSI_ERR_OOM;
  }
  c->B0 = box;
  fsi_status st = c->x.b0_method == 1 ? build_b0_columns(c) : build_b0(c);
  const double secs = c->b0_seconds;
  c->B0 = full;
  if (st == FSI_OK) {
    k_expand<<<1024, 256, 0, c->stream>>>(full, box, c->n_box, c->n_sd);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) st = FSI_ERR_CUDA;
  }
  ctx_dev_free(c, box);
  if (st != FSI_OK) return st;
  st = c->prec == FSI_PREC_FP64 ? app_columns_t<double>(c) : app_columns_t<float>(c);
  c->b0_seconds = secs;
  return st;
}

fsi_status launch_appended_source(fsi_ctx* c) {
  if (c->n_app == 0) return FSI_OK;
  const int ai0 = c->app_box[0], aj0 = c->app_box[1], ai1 = c->app_box[2], aj1 = c->app_box[3];
  // the window the sub-domain source kernel writes every step: Omega_0 grown by 3 cells, interior vertices
  const int si0 = std::max(c->i_lo - 3, 1), si1 = std::min(c->i_hi + 3, c->nx - 1);
  const int sj0 = std::max(c->j_lo - 3, 1), sj1 = std::min(c->j_hi + 3, c->ny - 1);
  const dim3 grid((unsigned)((ai1 - ai0 + 64) / 64), (unsigned)(aj1 - aj0 + 1));
  const double pre_h = c->ds / (c->g.h * c->g.h * c->g.h);
  if (c->prec == FSI_PREC_FP64)
    k_app_src<double><<<grid, 64, 0, c->stream>>>((double*)c->src, c->ps, ai0, aj0, ai1, aj1, si0, sj0, si1, sj1,
                                                  c->d_app_win, c->d_app_idx + c->nb, c->d_f, c->nb, c->n_app, pre_h);
  else
    k_app_src<float><<<grid, 64, 0, c->stream>>>((float*)c->src, c->ps, ai0, aj0, ai1, aj1, si0, sj0, si1, sj1,
                                                 c->d_app_win, c->d_app_idx + c->nb, c->d_f, c->nb, c->n_app, pre_h);
  FSI_CUDA_TRY(cudaGetLastError());
  c->launches_per_step += 1;
  return FSI_OK;
}
