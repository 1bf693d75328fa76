// Sparse B0' (Sec. 3.3; Eq. filtereq as each column is built, reading R8: keep b_ij with
// |b_ij| > eps |b_jj|) in a windowed column format.
//
// The entries of a column decay away from the column's own Omega_0 point (Sec. 3.3.1), and the decay is
// nearly the same for every column (near-translation invariance).  Each column j therefore stores one
// window of (2w+1) x (2w+1) Omega_0 points around its point, for both velocity components of the row:
//   W[j][ca][dj + w][di + w] = b'((ca, jb + dj, ib + di), j),  |dj|, |di| <= w,
// zero where the filter drops the entry or the point lies outside Omega_0 (for a union of boxes the window
// is taken in the bounding box, so columns near another box hold the cross-box entries), and a lookup of any entry is
// O(1).  w is the largest extent of a kept entry over all columns, found by a scan whose radius doubles
// until no kept entry touches its edge; B0' built this way equals the filter of the dense B0 entry by
// entry (the entries come from the same lattice Green's-function tables, in the same rounding order, as
// the dense build).
#include <chrono>
#include <cmath>
#include <vector>
#include "internal.h"

namespace {

__device__ __forceinline__ int block_max_int(int v, int* red) {
  v = __reduce_max_sync(0xffffffffu, v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  int r = 0;
  for (int k = 0; k < nw; ++k) r = max(r, red[k]);
  __syncthreads();
  return r;
}

// Omega_0 membership of box vertex (ia, ja): inside the box (or the union's bounding box) and, for a union,
// marked in its map.
__device__ __forceinline__ bool sd_member(const int* map, int ni, int nj, int ia, int ja) {
  if (ja < 0 || ja >= nj || ia < 0 || ia >= ni) return false;
  return !map || map[(long)ja * ni + ia] >= 0;
}

// One CTA per column: the largest |dj|, |di| of a kept entry within radius W (into ext[0], ext[1]).  bx is the
// box (or the bounding box of a union, with its map and point list) of the n_sd Omega_0 points.
__global__ void __launch_bounds__(256) k_window_extent(const double* __restrict__ tab, B0Box bx, int n_sd,
                                                       const int* __restrict__ map, const int* __restrict__ vert,
                                                       double eps, int W, int* ext) {
  __shared__ int red[32];
  const int ni = bx.ni, nj = bx.nj, nx2 = 2 * ni - 1;
  const long per = (long)nx2 * (2 * nj - 1);
  const int col = blockIdx.x, cb = col / n_sd, p = col - cb * n_sd;
  int ib, jb;
  sd_vertex(vert, ni, p, &ib, &jb);
  const double thr = eps * fabs(b0_entry(tab, per, nx2, ni, nj, cb, jb, ib, cb, jb, ib));
  const int side = 2 * W + 1, area = side * side;
  int mj = 0, mi = 0;
  for (int e = threadIdx.x; e < 2 * area; e += blockDim.x) {
    const int ca = e / area, r = e - ca * area, dj = r / side - W, di = r - (r / side) * side - W;
    const int ja = jb + dj, ia = ib + di;
    if (!sd_member(map, ni, nj, ia, ja)) continue;
    if (fabs(b0_entry(tab, per, nx2, ni, nj, ca, ja, ia, cb, jb, ib)) > thr) {
      mj = max(mj, abs(dj));
      mi = max(mi, abs(di));
    }
  }
  mj = block_max_int(mj, red);
  mi = block_max_int(mi, red);
  if (threadIdx.x == 0) {
    atomicMax(ext, mj);
    atomicMax(ext + 1, mi);
  }
}

// One CTA per column: its window (zero where dropped or outside Omega_0); kept entries counted in nnz.
__global__ void __launch_bounds__(256) k_fill_window(double* __restrict__ Wv, const double* __restrict__ tab,
                                                     B0Box bx, int n_sd, const int* __restrict__ map,
                                                     const int* __restrict__ vert, double eps, int w,
                                                     unsigned long long* nnz) {
  __shared__ int red[32];
  const int ni = bx.ni, nj = bx.nj, nx2 = 2 * ni - 1;
  const long per = (long)nx2 * (2 * nj - 1);
  const int col = blockIdx.x, cb = col / n_sd, p = col - cb * n_sd;
  int ib, jb;
  sd_vertex(vert, ni, p, &ib, &jb);
  const double thr = eps * fabs(b0_entry(tab, per, nx2, ni, nj, cb, jb, ib, cb, jb, ib));
  const int side = 2 * w + 1, area = side * side;
  double* out = Wv + (long)col * 2 * area;
  int kept = 0;
  for (int e = threadIdx.x; e < 2 * area; e += blockDim.x) {
    const int ca = e / area, r = e - ca * area, dj = r / side - w, di = r - (r / side) * side - w;
    const int ja = jb + dj, ia = ib + di;
    double v = 0.0;
    if (sd_member(map, ni, nj, ia, ja)) {
      v = b0_entry(tab, per, nx2, ni, nj, ca, ja, ia, cb, jb, ib);
      if (!(fabs(v) > thr)) v = 0.0;
      else ++kept;
    }
    out[e] = v;
  }
  kept = __reduce_add_sync(0xffffffffu, kept);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = kept;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += (unsigned long long)red[k];
    atomicAdd(nnz, s);
  }
}

__global__ void k_window_entries(const double* __restrict__ Wv, int w, int ni, int n_sd, const int64_t* rows,
                                 const int64_t* cols, int n, const int* __restrict__ vert, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[k] = b0w_lookup(Wv, w, ni, n_sd, rows[k], cols[k], vert);
}

}  // namespace

fsi_status build_b0_window(fsi_ctx* c, double drop_tol) {
  auto t0 = std::chrono::steady_clock::now();
  std::vector<B0Box> one(1, ctx_box(c));
  b0_layout(one);
  double* d_tab = nullptr;
  fsi_status st = b0_green_tables(c, one, &d_tab);
  if (st != FSI_OK) return st;
  const B0Box bx = one[0];
  const int n2 = 2 * c->n_sd;
  int* d_ext = nullptr;
  unsigned long long* d_nnz = nullptr;
  do {
    if (ctx_dev_malloc(c, (void**)&d_ext, 2 * sizeof(int)) != cudaSuccess ||
        ctx_dev_malloc(c, (void**)&d_nnz, sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      st = FSI_ERR_OOM;
      break;
    }
    const int wmax = bx.ni > bx.nj ? bx.ni : bx.nj;
    int W = 16 < wmax ? 16 : wmax, w = 0;
    for (;;) {  // scan radius doubles while a kept entry touches the edge of the scanned window
      int ext[2] = {0, 0};
      if (cudaMemcpyAsync(d_ext, ext, sizeof(ext), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
        st = FSI_ERR_CUDA;
        break;
      }
      k_window_extent<<<n2, 256, 0, c->stream>>>(d_tab, bx, c->n_sd, c->d_sd_map, c->d_sd_vert, drop_tol, W, d_ext);
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpyAsync(ext, d_ext, sizeof(ext), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        st = FSI_ERR_CUDA;
        break;
      }
      w = ext[0] > ext[1] ? ext[0] : ext[1];
      if (w < W || W >= wmax) break;
      W = 2 * W < wmax ? 2 * W : wmax;
    }
    if (st != FSI_OK) break;
    if (w < 1) w = 1;
    const long area = (long)(2 * w + 1) * (2 * w + 1);
    if (!(c->Bw = (double*)ctx_alloc(c, (size_t)n2 * 2 * area * sizeof(double)))) {
      st = FSI_ERR_OOM;
      break;
    }
    if (cudaMemsetAsync(d_nnz, 0, sizeof(unsigned long long), c->stream) != cudaSuccess) {
      st = FSI_ERR_CUDA;
      break;
    }
    k_fill_window<<<n2, 256, 0, c->stream>>>(c->Bw, d_tab, bx, c->n_sd, c->d_sd_map, c->d_sd_vert, drop_tol, w, d_nnz);
    unsigned long long nnz = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&nnz, d_nnz, sizeof(nnz), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      st = FSI_ERR_CUDA;
      break;
    }
    c->bw = w;
    c->b0_nnz = (long long)nnz;
  } while (0);
  ctx_dev_free(c, d_tab);
  ctx_dev_free(c, d_ext);
  ctx_dev_free(c, d_nnz);
  c->b0_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

fsi_status b0_window_entries(fsi_ctx* c, const int64_t* d_rows, const int64_t* d_cols, int n, double* d_out) {
  k_window_entries<<<(n + 255) / 256, 256, 0, c->stream>>>(c->Bw, c->bw, c->ni, c->n_sd, d_rows, d_cols, n,
                                                           c->d_sd_vert, d_out);
  return cudaGetLastError() == cudaSuccess ? FSI_OK : FSI_ERR_CUDA;
}
