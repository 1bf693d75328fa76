// Double-precision Cholesky factor of the shifted sub-domain matrix, L L^T = B0 + tau I.
//
// B0 is only positive semi-definite when Omega_0 is sampled at the flow-grid spacing (the E0 C rows of
// neighbouring points are nearly dependent), so the factor is taken of B0 + tau I with
// tau = tau_rel * max_i B0_ii.  Blocked right-looking algorithm with 64-wide panels:
//   1. k_potrf_diag: the 64 x 64 diagonal block, one CTA, in shared memory;
//   2. k_trsm_panel: rows below solve X L_kk^T = A_ik, one thread per row, L_kk in shared memory;
//   3. k_syrk_lower: trailing update A_22 -= L_21 L_21^T on 64 x 64 lower-triangle tiles, 4 x 4 outputs
//      per thread from shared-memory panels.
// All arithmetic is double; on this part the FP64 units bound it (n^3/3 flops).
#include <chrono>
#include <cmath>
#include "internal.h"

namespace {

constexpr int NB = 64;

__global__ void k_shift_copy(double* __restrict__ L, const double* __restrict__ B0, long n, double tau) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const long i = e / n, j = e - i * n;
  L[e] = j <= i ? B0[e] + (i == j ? tau : 0.0) : 0.0;
}

__global__ void k_max_diag(const double* __restrict__ B0, long n, double* out) {
  __shared__ double red[256];
  double m = 0.0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, B0[i * n + i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Cholesky of the diagonal block at (k0, k0) of size b <= NB, in place (lower).
__global__ void __launch_bounds__(256) k_potrf_diag(double* __restrict__ L, long n, long k0, int b, int* status) {
  __shared__ double A[NB][NB + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    A[i][j] = j <= i ? L[(k0 + i) * n + k0 + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      const double d = A[j][j];
      if (!(d > 0.0)) {
        dev_set_status(status, FSI_ERR_NONFINITE);
        A[j][j] = 1.0;
      } else {
        A[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    const double djj = A[j][j];
    for (int i = j + 1 + tid; i < b; i += blockDim.x) A[i][j] /= djj;
    __syncthreads();
    const int m = b - j - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, c = j + 1 + e % m;
      if (c <= i) A[i][c] -= A[i][j] * A[c][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    if (j <= i) L[(k0 + i) * n + k0 + j] = A[i][j];
  }
}

// Rows r >= k0 + b: L[r][k0..k0+b) <- A[r][k0..k0+b) L_kk^{-T}.  64 rows per CTA, one thread per row.
__global__ void __launch_bounds__(64) k_trsm_panel(double* __restrict__ L, long n, long k0, int b) {
  extern __shared__ double dsm[];  // two NB x (NB + 1) tiles
  double(*D)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(dsm);
  double(*R)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(dsm + NB * (NB + 1));
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    D[i][j] = j <= i ? L[(k0 + i) * n + k0 + j] : 0.0;
  }
  const long r0 = k0 + b + (long)blockIdx.x * NB;
  for (int e = tid; e < NB * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    R[i][j] = (r0 + i < n) ? L[(r0 + i) * n + k0 + j] : 0.0;
  }
  __syncthreads();
  if (r0 + tid < n) {
    for (int c = 0; c < b; ++c) {
      double v = R[tid][c];
      for (int cc = 0; cc < c; ++cc) v -= R[tid][cc] * D[c][cc];
      R[tid][c] = v / D[c][c];
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * b; e += blockDim.x) {
    const int i = e / b, j = e - i * b;
    if (r0 + i < n) L[(r0 + i) * n + k0 + j] = R[i][j];
  }
}

// Trailing update on lower-triangle tiles (ti >= tj) of the matrix from t0 on: C -= L_i L_j^T over the panel.
__global__ void __launch_bounds__(256) k_syrk_lower(double* __restrict__ L, long n, long k0, int b, long t0) {
  extern __shared__ double dsm[];  // two NB x (NB + 1) panels
  double(*Pi)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(dsm);
  double(*Pj)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(dsm + NB * (NB + 1));
  // tile index -> (ti, tj) with tj <= ti
  const long t = blockIdx.x;
  long ti = (long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  if (ti * (ti + 1) / 2 > t) --ti;
  if ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  const long tj = t - ti * (ti + 1) / 2;
  const long ri = t0 + ti * NB, rj = t0 + tj * NB;
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * b; e += blockDim.x) {
    const int i = e / b, c = e - i * b;
    Pi[i][c] = (ri + i < n) ? L[(ri + i) * n + k0 + c] : 0.0;
    Pj[i][c] = (rj + i < n) ? L[(rj + i) * n + k0 + c] : 0.0;
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads, 4 x 4 outputs each (rows ty + 16 q)
  double acc[4][4] = {};
  for (int c = 0; c < b; ++c) {
    double a[4], bb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = Pi[ty + 16 * q][c];
      bb[q] = Pj[tx + 16 * q][c];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int p = 0; p < 4; ++p) acc[q][p] += a[q] * bb[p];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const long i = ri + ty + 16 * q, j = rj + tx + 16 * p;
      if (i < n && j < n && j <= i) L[i * n + j] -= acc[q][p];
    }
}

}  // namespace

extern "C" fsi_status fsi_factor_operator(fsi_ctx* c, double tau_rel, double* tau_out, double* seconds) {
  if (!c || tau_rel < 0) return FSI_ERR_INVALID_ARG;
  if (!c->have_b0) return FSI_ERR_STATE;
  if (!c->B0) return FSI_ERR_UNSUPPORTED;  // the sparse B0' is not factored
  const long n = 2L * c->n_sd;
  auto t0 = std::chrono::steady_clock::now();
  if (!c->d_factor) {
    c->d_factor = (double*)ctx_alloc(c, (size_t)n * n * sizeof(double));
    if (!c->d_factor) return FSI_ERR_OOM;
  }
  double* d_max = nullptr;
  FSI_CUDA_TRY(ctx_dev_malloc(c, (void**)&d_max, sizeof(double)));
  k_max_diag<<<1, 256, 0, c->stream>>>(c->B0, n, d_max);
  double dmax = 0.0;
  cudaError_t e = cudaMemcpyAsync(&dmax, d_max, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  ctx_dev_free(c, d_max);
  FSI_CUDA_TRY(e);
  const double tau = tau_rel * dmax;
  const size_t sm2 = (size_t)2 * NB * (NB + 1) * sizeof(double);
  cudaFuncSetAttribute(k_trsm_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  cudaFuncSetAttribute(k_syrk_lower, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  k_shift_copy<<<(unsigned)((n * n + 255) / 256), 256, 0, c->stream>>>(c->d_factor, c->B0, n, tau);
  for (long k0 = 0; k0 < n; k0 += NB) {
    const int b = (int)(n - k0 < NB ? n - k0 : NB);
    k_potrf_diag<<<1, 256, 0, c->stream>>>(c->d_factor, n, k0, b, c->d_status);
    const long rem = n - k0 - b;
    if (rem <= 0) break;
    k_trsm_panel<<<(unsigned)((rem + NB - 1) / NB), 64, sm2, c->stream>>>(c->d_factor, n, k0, b);
    const long nt = (rem + NB - 1) / NB;
    k_syrk_lower<<<(unsigned)(nt * (nt + 1) / 2), 256, sm2, c->stream>>>(c->d_factor, n, k0, b, k0 + b);
  }
  FSI_CUDA_TRY(cudaGetLastError());
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (tau_out) *tau_out = tau;
  if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int st = 0;
  FSI_CUDA_TRY(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  return (fsi_status)st;
}

__global__ static void k_gather_factor(const double* L, long n2, const int64_t* rows, const int64_t* cols, int n,
                                       double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = L[rows[k] * n2 + cols[k]];
}

extern "C" fsi_status fsi_get_factor_entries(fsi_ctx* c, const int64_t* rows, const int64_t* cols, int n,
                                             double* out) {
  if (!c || n < 0 || (n > 0 && (!rows || !cols || !out))) return FSI_ERR_INVALID_ARG;
  if (!c->d_factor) return FSI_ERR_STATE;
  const long n2 = 2L * c->n_sd;
  for (int k = 0; k < n; ++k)
    if (rows[k] < 0 || rows[k] >= n2 || cols[k] < 0 || cols[k] >= n2) return FSI_ERR_INVALID_ARG;
  if (n == 0) return FSI_OK;
  int64_t *dr = nullptr, *dc = nullptr;
  double* dout = nullptr;
  fsi_status st = FSI_OK;
  if (ctx_dev_malloc(c, (void**)&dr, n * 8) != cudaSuccess || ctx_dev_malloc(c, (void**)&dc, n * 8) != cudaSuccess ||
      ctx_dev_malloc(c, (void**)&dout, n * 8) != cudaSuccess) {
    st = FSI_ERR_OOM;
  } else if (cudaMemcpyAsync(dr, rows, n * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
             cudaMemcpyAsync(dc, cols, n * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
    st = FSI_ERR_CUDA;
  } else {
    k_gather_factor<<<(n + 255) / 256, 256, 0, c->stream>>>(c->d_factor, n2, dr, dc, n, dout);
    if (cudaMemcpyAsync(out, dout, n * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      st = FSI_ERR_CUDA;
  }
  ctx_dev_free(c, dr);
  ctx_dev_free(c, dc);
  ctx_dev_free(c, dout);
  return st;
}
