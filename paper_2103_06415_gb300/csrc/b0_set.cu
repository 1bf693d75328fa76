// B0 for several independent Omega_0 boxes on one grid, built together (fsi_b0_set_* in ibfsi.h).
// A one-level context supplies the grid tables and the column-solve machinery; the matrices of all boxes
// live in one device allocation, box after box.
#include <chrono>
#include <new>
#include <vector>
#include "internal.h"

struct fsi_b0_set {
  fsi_ctx* c;
  std::vector<B0Box> boxes;
  std::vector<int> i_hi, j_hi;
  double* d_out;
  double seconds;
};

__global__ static void k_gather_set(const double* M, long n2, const int64_t* rows, const int64_t* cols, int n,
                                    double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = M[rows[k] * n2 + cols[k]];
}

extern "C" fsi_status fsi_b0_set_build(const fsi_grid_desc* grid, const fsi_exec_desc* exec, const fsi_box* boxes,
                                       int n_boxes, fsi_b0_set** out) {
  if (!grid || !exec || !boxes || !out || n_boxes < 1 || n_boxes > 4096) return FSI_ERR_INVALID_ARG;
  *out = nullptr;
  if (exec->b0_method != 0 && exec->b0_method != 1) return FSI_ERR_INVALID_ARG;
  fsi_grid_desc g1 = *grid;
  g1.n_levels = 1;
  fsi_b0_set* s = new (std::nothrow) fsi_b0_set();
  if (!s) return FSI_ERR_OOM;
  for (int k = 0; k < n_boxes; ++k) {
    int i_lo, i_hi, j_lo, j_hi;
    const fsi_status st = snap_box(g1, boxes[k], &i_lo, &i_hi, &j_lo, &j_hi);
    if (st != FSI_OK) {
      delete s;
      return st;
    }
    B0Box b = {};
    b.i_lo = i_lo;
    b.j_lo = j_lo;
    b.ni = i_hi - i_lo + 1;
    b.nj = j_hi - j_lo + 1;
    s->boxes.push_back(b);
    s->i_hi.push_back(i_hi);
    s->j_hi.push_back(j_hi);
  }
  fsi_status st = fsi_create(&g1, exec, &s->c);
  if (st != FSI_OK) {
    delete s;
    return st;
  }
  const long entries = b0_layout(s->boxes);
  auto t0 = std::chrono::steady_clock::now();
  if (!(s->d_out = (double*)ctx_alloc(s->c, (size_t)entries * 8))) {
    st = FSI_ERR_OOM;
  } else {
    st = exec->b0_method == 1 ? b0_columns(s->c, s->boxes, s->d_out) : b0_green(s->c, s->boxes, s->d_out);
  }
  s->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (st != FSI_OK) {
    fsi_b0_set_destroy(s);
    return st;
  }
  *out = s;
  return FSI_OK;
}

extern "C" fsi_status fsi_b0_set_box(const fsi_b0_set* s, int box, int* i_lo, int* i_hi, int* j_lo, int* j_hi,
                                     int* n_sd) {
  if (!s || box < 0 || box >= (int)s->boxes.size()) return FSI_ERR_INVALID_ARG;
  const B0Box& b = s->boxes[box];
  if (i_lo) *i_lo = b.i_lo;
  if (i_hi) *i_hi = s->i_hi[box];
  if (j_lo) *j_lo = b.j_lo;
  if (j_hi) *j_hi = s->j_hi[box];
  if (n_sd) *n_sd = b.n_sd;
  return FSI_OK;
}

extern "C" fsi_status fsi_b0_set_entries(fsi_b0_set* s, int box, const int64_t* rows, const int64_t* cols, int n,
                                         double* out) {
  if (!s || box < 0 || box >= (int)s->boxes.size() || n < 0 || (n > 0 && (!rows || !cols || !out)))
    return FSI_ERR_INVALID_ARG;
  const B0Box& b = s->boxes[box];
  const long n2 = 2L * b.n_sd;
  for (int k = 0; k < n; ++k)
    if (rows[k] < 0 || rows[k] >= n2 || cols[k] < 0 || cols[k] >= n2) return FSI_ERR_INVALID_ARG;
  if (n == 0) return FSI_OK;
  cudaStream_t st_ = s->c->stream;
  int64_t *dr = nullptr, *dc = nullptr;
  double* dout = nullptr;
  fsi_status st = FSI_OK;
  if (ctx_dev_malloc(s->c, (void**)&dr, n * 8) != cudaSuccess || ctx_dev_malloc(s->c, (void**)&dc, n * 8) != cudaSuccess ||
      ctx_dev_malloc(s->c, (void**)&dout, n * 8) != cudaSuccess) {
    cudaGetLastError();
    st = FSI_ERR_OOM;
  } else if (cudaMemcpyAsync(dr, rows, n * 8, cudaMemcpyHostToDevice, st_) != cudaSuccess ||
             cudaMemcpyAsync(dc, cols, n * 8, cudaMemcpyHostToDevice, st_) != cudaSuccess) {
    st = FSI_ERR_CUDA;
  } else {
    k_gather_set<<<(n + 255) / 256, 256, 0, st_>>>(s->d_out + b.out_off, n2, dr, dc, n, dout);
    if (cudaMemcpyAsync(out, dout, n * 8, cudaMemcpyDeviceToHost, st_) != cudaSuccess ||
        cudaStreamSynchronize(st_) != cudaSuccess)
      st = FSI_ERR_CUDA;
  }
  ctx_dev_free(s->c, dr);
  ctx_dev_free(s->c, dc);
  ctx_dev_free(s->c, dout);
  return st;
}

extern "C" fsi_status fsi_b0_set_stats(const fsi_b0_set* s, double* seconds, size_t* device_bytes) {
  if (!s) return FSI_ERR_INVALID_ARG;
  if (seconds) *seconds = s->seconds;
  if (device_bytes) *device_bytes = s->c->dev_bytes;
  return FSI_OK;
}

extern "C" void fsi_b0_set_destroy(fsi_b0_set* s) {
  if (!s) return;
  fsi_destroy(s->c);
  delete s;
}
