// Offline stage (Algorithm 1, Eq. action): B0 = E0 C (C^T A C)^{-1} C^T E0^T on the finest level with
// homogeneous boundary values, dense, in double.
//
// Instead of one 2-D solve per column, every column is produced at once from the lattice Green's function
// of M = (C^T A C)^{-1} = Lap^{-1} A_w^{-1}.  With the DST-I eigen-decomposition of Sec. 3.2.1,
//   M[(i,j),(i',j')] = g(i-i', j-j') - g(i+i', j-j') - g(i-i', j+j') + g(i+i', j+j'),
//   g(p, q) = 1/(Mx My) sum_{k,l} d_kl cos(pi k p/Mx) cos(pi l q/My),  d_kl = 1/(lambda_kl a_kl),
// (product-to-sum of the sine eigenvectors), so M is Toeplitz-minus-Hankel in each direction.  A row of
// E0 C is a 6-vertex stencil (u: w_dx (s[j+1] - s[j-1])/2h; v: -w_dy (s[i+1] - s[i-1])/2h), hence
//   B0[a][b] = T--(ia-ib, ja-jb) - T+-(ia+ib, ja-jb) - T-+(ia-ib, ja+jb) + T++(ia+ib, ja+jb)
// with 16 small tables (4 component blocks x 4 image terms) of stencil-convolved g.  The result equals the
// column-by-column definition up to rounding order; the cost is one pass writing B0 plus two small
// cosine contractions for g.
#include <chrono>
#include <cmath>
#include <vector>
#include "internal.h"

namespace {

// T1[k][q] = sum_l d_kl cos(pi l q / My), k = 1..Nx (row k-1), q = 0..My
__global__ void k_g_stage1(double* __restrict__ T1, int Nx, int Ny, int My, const double* __restrict__ lx,
                           const double* __restrict__ ly, const double* __restrict__ cy, double inv_h2,
                           double inv_dt, double inv_2re) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y + 1;
  if (q > My) return;
  const int period = 2 * My;
  double acc = 0.0;
  int idx = 0;  // (l*q) mod 2My, incremented
  for (int l = 1; l <= Ny; ++l) {
    idx += q;
    if (idx >= period) idx -= period;
    const double lam = (lx[k] + ly[l]) * inv_h2;
    const double a = inv_dt + lam * inv_2re;
    acc += cy[idx] / (lam * a);
  }
  T1[(long)(k - 1) * (My + 1) + q] = acc;
}

// g[p][q] = norm * sum_k cos(pi k p/Mx) T1[k][q], p = 0..Mx, q = 0..My
__global__ void k_g_stage2(double* __restrict__ g, const double* __restrict__ T1, int Nx, int Mx, int My,
                           const double* __restrict__ cx, double norm) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (q > My) return;
  const int period = 2 * Mx;
  double acc = 0.0;
  int idx = 0;
  for (int k = 1; k <= Nx; ++k) {
    idx += p;
    if (idx >= period) idx -= period;
    acc += cx[idx] * T1[(long)(k - 1) * (My + 1) + q];
  }
  g[(long)p * (My + 1) + q] = norm * acc;
}

__device__ __forceinline__ int fold(int p, int M) {
  int a = p < 0 ? -p : p;
  a %= 2 * M;
  return a > M ? 2 * M - a : a;
}

struct Stencil {
  int n;
  int dx[6], dy[6];
  double w[6];
};

__device__ void make_stencil(int comp, double h, Stencil* s) {
  const double w3[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
  s->n = 6;
  int t = 0;
  for (int d = -1; d <= 1; ++d)
    for (int e = -1; e <= 1; e += 2) {
      if (comp == 0) {  // u = sum_d w_d (s[j+1][i+d] - s[j-1][i+d]) / (2h)
        s->dx[t] = d;
        s->dy[t] = e;
        s->w[t] = w3[d + 1] * (double)e / (2.0 * h);
      } else {  // v = -sum_d w_d (s[j+d][i+1] - s[j+d][i-1]) / (2h)
        s->dx[t] = e;
        s->dy[t] = d;
        s->w[t] = -w3[d + 1] * (double)e / (2.0 * h);
      }
      ++t;
    }
}

// tables[((ca*2+cb)*4 + term)][iy][ix] (x index contiguous), term bit0: x uses the sum index, bit1: y uses
// the sum index
__global__ void k_tables(double* __restrict__ tab, const double* __restrict__ g, int Mx, int My, int ni, int nj,
                         int i_lo, int j_lo, double h) {
  const int nx2 = 2 * ni - 1, ny2 = 2 * nj - 1;
  const long per = (long)nx2 * ny2;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 16 * per) return;
  const int tb = (int)(e / per);
  const long r = e - (long)tb * per;
  const int iy = (int)(r / nx2), ix = (int)(r - (long)iy * nx2);
  const int term = tb & 3, cab = tb >> 2, ca = cab >> 1, cb = cab & 1;
  Stencil sa, sb;
  make_stencil(ca, h, &sa);
  make_stencil(cb, h, &sb);
  const bool xs = term & 1, ys = term & 2;
  const int X = xs ? ix + 2 * i_lo : ix - (ni - 1);
  const int Y = ys ? iy + 2 * j_lo : iy - (nj - 1);
  double acc = 0.0;
  for (int u = 0; u < 6; ++u)
    for (int v = 0; v < 6; ++v) {
      const int px = xs ? X + sa.dx[u] + sb.dx[v] : X + sa.dx[u] - sb.dx[v];
      const int py = ys ? Y + sa.dy[u] + sb.dy[v] : Y + sa.dy[u] - sb.dy[v];
      acc += sa.w[u] * sb.w[v] * g[(long)fold(px, Mx) * (My + 1) + fold(py, My)];
    }
  tab[e] = acc;
}

// One CTA per row a of B0: B0[a][b] = T--(ia-ib, ja-jb) - T+-(ia+ib, ja-jb) - T-+(ia-ib, ja+jb)
// + T++(ia+ib, ja+jb); threads run along ib so stores and table reads are contiguous.
__global__ void __launch_bounds__(256) k_fill(double* __restrict__ B0, const double* __restrict__ tab, int ni,
                                              int nj, int n_sd) {
  const long n2 = 2L * n_sd;
  const int nx2 = 2 * ni - 1, ny2 = 2 * nj - 1;
  const long per = (long)nx2 * ny2;
  for (long a = blockIdx.x; a < n2; a += gridDim.x) {
    const int ca = (int)(a / n_sd);
    const int pa = (int)(a - (long)ca * n_sd);
    const int ja = pa / ni, ia = pa - ja * ni;
    double* row = B0 + a * n2;
    for (int cb = 0; cb < 2; ++cb) {
      const double* t = tab + (long)((ca * 2 + cb) * 4) * per;
      for (int jb = 0; jb < nj; ++jb) {
        const double* tmm = t + (long)(ja - jb + nj - 1) * nx2;
        const double* tpm = t + per + (long)(ja - jb + nj - 1) * nx2;
        const double* tmp = t + 2 * per + (long)(ja + jb) * nx2;
        const double* tpp = t + 3 * per + (long)(ja + jb) * nx2;
        double* out = row + (long)cb * n_sd + (long)jb * ni;
        for (int ib = threadIdx.x; ib < ni; ib += blockDim.x) {
          const int D = ia - ib + ni - 1, S = ia + ib;
          out[ib] = tmm[D] - tpm[S] - tmp[D] + tpp[S];
        }
      }
    }
  }
}

}  // namespace

fsi_status build_b0(fsi_ctx* c) {
  auto t0 = std::chrono::steady_clock::now();
  const int Nx = c->Nx, Ny = c->Ny, Mx = c->Mx, My = c->My;
  const double h = c->g.h;
  std::vector<double> cx(2 * Mx), cy(2 * My);
  for (int p = 0; p < 2 * Mx; ++p) cx[p] = std::cos(M_PI * (double)p / (double)Mx);
  for (int q = 0; q < 2 * My; ++q) cy[q] = std::cos(M_PI * (double)q / (double)My);
  double *d_cx = nullptr, *d_cy = nullptr, *d_T1 = nullptr, *d_g = nullptr, *d_tab = nullptr;
  const int nx2 = 2 * c->ni - 1, ny2 = 2 * c->nj - 1;
  const size_t tab_n = (size_t)16 * nx2 * ny2;
  fsi_status st = FSI_OK;
  do {
    if (cudaMalloc(&d_cx, cx.size() * 8) != cudaSuccess || cudaMalloc(&d_cy, cy.size() * 8) != cudaSuccess ||
        cudaMalloc(&d_T1, (size_t)Nx * (My + 1) * 8) != cudaSuccess ||
        cudaMalloc(&d_g, (size_t)(Mx + 1) * (My + 1) * 8) != cudaSuccess ||
        cudaMalloc(&d_tab, tab_n * 8) != cudaSuccess) {
      st = FSI_ERR_OOM;
      break;
    }
    if (cudaMemcpyAsync(d_cx, cx.data(), cx.size() * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(d_cy, cy.data(), cy.size() * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
      st = FSI_ERR_CUDA;
      break;
    }
    k_g_stage1<<<dim3((My + 1 + 127) / 128, Nx), 128, 0, c->stream>>>(d_T1, Nx, Ny, My, c->lx, c->ly, d_cy,
                                                                      1.0 / (h * h), 1.0 / c->g.dt, 0.5 / c->g.re);
    k_g_stage2<<<dim3((My + 1 + 127) / 128, Mx + 1), 128, 0, c->stream>>>(d_g, d_T1, Nx, Mx, My, d_cx,
                                                                          1.0 / ((double)Mx * (double)My));
    k_tables<<<(unsigned)((tab_n + 127) / 128), 128, 0, c->stream>>>(d_tab, d_g, Mx, My, c->ni, c->nj, c->i_lo,
                                                                     c->j_lo, h);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
    k_fill<<<nsm * 16, 256, 0, c->stream>>>(c->B0, d_tab, c->ni, c->nj, c->n_sd);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) st = FSI_ERR_CUDA;
  } while (0);
  cudaFree(d_cx);
  cudaFree(d_cy);
  cudaFree(d_T1);
  cudaFree(d_g);
  cudaFree(d_tab);
  c->b0_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st;
}
