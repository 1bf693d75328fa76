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
// column-by-column definition up to rounding order; the cost is one pass writing B0 plus the two cosine
// sums of g, each a batch of DCT-I rows done by FFT in double.  g depends on the grid only, so several
// Omega_0 boxes on one grid share it and their tables and matrices are produced by one launch of each
// kernel.
#include <chrono>
#include <cmath>
#include <mutex>
#include <vector>
#include "dst.cuh"
#include "internal.h"

namespace {

// DCT-I rows by FFT: out[r][q] = scale * sum_{l=1}^{M-1} x_r[l] cos(pi l q / M), q = 0..M.  The even
// extension y (y[l] = y[2M-l] = x_r[l], y[0] = y[M] = 0) has the real DFT Y_q = 2 sum_l x_r[l] cos(pi l q/M),
// so two rows packed as y_a + i y_b give Y_a = Re Z, Y_b = Im Z of one complex FFT of length L = 2M.
// Rows come from `in` (element (r, l) at in[r*in_rs + (l-1)*in_es]) or, when in == NULL, from the spectral
// Green's-function weights d_kl = 1/(lambda_kl a_kl) with k = r+1 (the first cosine sum of g).
template <int PER, int R3 = 1>
__global__ void __launch_bounds__(256) k_dct1(const double* __restrict__ in, long in_rs, long in_es, int nrows,
                                              int M, double* __restrict__ out, long out_rs, long out_es,
                                              const double2* __restrict__ tw, int logL, double scale,
                                              const double* __restrict__ lx, const double* __restrict__ ly,
                                              double inv_h2, double inv_dt, double inv_2re) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* buf = reinterpret_cast<double2*>(smem_raw);
  const int L = R3 << logL;  // logL: log2 of the power-of-two part
  const double2* tws = dst::stage_twiddles<double>(buf + L, tw, L, (size_t)2 * L * sizeof(double2));
  const int r0 = 2 * blockIdx.x;
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    const int ll = l <= M ? l : L - l;
    double a = 0.0, b = 0.0;
    if (ll >= 1 && ll <= M - 1) {
      for (int e = 0; e < 2; ++e) {
        const int r = r0 + e;
        double v = 0.0;
        if (r < nrows) {
          if (in) {
            v = in[(long)r * in_rs + (long)(ll - 1) * in_es];
          } else {
            const double lam = (lx[r + 1] + ly[ll]) * inv_h2;
            v = 1.0 / (lam * (inv_dt + lam * inv_2re));
          }
        }
        if (e == 0) a = v;
        else b = v;
      }
    }
    buf[l] = make_double2(a, b);
  }
  __syncthreads();
  dst::block_fft<double, PER, R3>(buf, L, logL, tws);
  for (int q = threadIdx.x; q <= M; q += blockDim.x) {
    const double2 z = buf[q];
    if (r0 < nrows) out[(long)r0 * out_rs + (long)q * out_es] = 0.5 * scale * z.x;
    if (r0 + 1 < nrows) out[(long)(r0 + 1) * out_rs + (long)q * out_es] = 0.5 * scale * z.y;
  }
}

// launch: one CTA per row pair, 2^logP / (4 PER) threads (one complex row of length L = r3 2^logP per CTA)
fsi_status launch_dct1(const double* in, long in_rs, long in_es, int nrows, int M, double* out, long out_rs,
                       long out_es, const double2* tw, int L, double scale, const double* lx, const double* ly,
                       double inv_h2, double inv_dt, double inv_2re, cudaStream_t st) {
  int logL = 0, r3 = 1;
  if (!dst::split_length(L, &logL, &r3)) return FSI_ERR_UNSUPPORTED;
  const int P = 1 << logL;
  const int nthr = P / 4 < 256 ? P / 4 : 256;
  const int per = P / (4 * nthr);
  const size_t sm = dst::pass_smem<double>((size_t)L, L);
  const dim3 grid((nrows + 1) / 2);
  static std::once_flag attrs;  // contexts may be built on several host threads (the server's worker)
  std::call_once(attrs, [] {
    cudaFuncSetAttribute(k_dct1<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_dct1<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_dct1<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_dct1<1, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_dct1<2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (r3 == 3) {
    if (per == 1) k_dct1<1, 3><<<grid, nthr, sm, st>>>(in, in_rs, in_es, nrows, M, out, out_rs, out_es, tw, logL, scale, lx, ly, inv_h2, inv_dt, inv_2re);
    else if (per == 2) k_dct1<2, 3><<<grid, nthr, sm, st>>>(in, in_rs, in_es, nrows, M, out, out_rs, out_es, tw, logL, scale, lx, ly, inv_h2, inv_dt, inv_2re);
    else return FSI_ERR_UNSUPPORTED;
    return cudaGetLastError() == cudaSuccess ? FSI_OK : FSI_ERR_CUDA;
  }
  switch (per) {
    case 1: k_dct1<1><<<grid, nthr, sm, st>>>(in, in_rs, in_es, nrows, M, out, out_rs, out_es, tw, logL, scale, lx, ly, inv_h2, inv_dt, inv_2re); break;
    case 2: k_dct1<2><<<grid, nthr, sm, st>>>(in, in_rs, in_es, nrows, M, out, out_rs, out_es, tw, logL, scale, lx, ly, inv_h2, inv_dt, inv_2re); break;
    case 4: k_dct1<4><<<grid, nthr, sm, st>>>(in, in_rs, in_es, nrows, M, out, out_rs, out_es, tw, logL, scale, lx, ly, inv_h2, inv_dt, inv_2re); break;
    default: return FSI_ERR_UNSUPPORTED;
  }
  return cudaGetLastError() == cudaSuccess ? FSI_OK : FSI_ERR_CUDA;
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

// Per box: tables[((ca*2+cb)*4 + term)][iy][ix] (x index contiguous), term bit0: x uses the sum index,
// bit1: y uses the sum index.  blockIdx.y is the box.
__global__ void k_tables(double* __restrict__ tab, const B0Box* __restrict__ bx, const double* __restrict__ g,
                         int Mx, int My, double h) {
  const B0Box b = bx[blockIdx.y];
  const int ni = b.ni, nj = b.nj;
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
  const int X = xs ? ix + 2 * b.i_lo : ix - (ni - 1);
  const int Y = ys ? iy + 2 * b.j_lo : iy - (nj - 1);
  double acc = 0.0;
  for (int u = 0; u < 6; ++u)
    for (int v = 0; v < 6; ++v) {
      const int px = xs ? X + sa.dx[u] + sb.dx[v] : X + sa.dx[u] - sb.dx[v];
      const int py = ys ? Y + sa.dy[u] + sb.dy[v] : Y + sa.dy[u] - sb.dy[v];
      acc += sa.w[u] * sb.w[v] * g[(long)fold(px, Mx) * (My + 1) + fold(py, My)];
    }
  tab[b.tab_off + e] = acc;
}

// One CTA per (box, ca, ja, cb, jb): the ni x ni block B0[(ca, ja, ia)][(cb, jb, ib)].  With
// r1 = ja - jb + nj - 1, r2 = ja + jb, D = ia - ib + ni - 1, S = ia + ib:
//   B0 = (T--[r1][D] - T-+[r2][D]) - (T+-[r1][S] - T++[r2][S]) = U[D] - V[S],
// U and V built once per block in shared memory, so each entry costs one FP64 subtraction (FP64 throughput
// per SM is low on sm_103; the block then writes at HBM speed).  blockIdx.x runs over the blocks of all
// boxes (blk_off = prefix sums of 4 nj^2).
__global__ void __launch_bounds__(256) k_fill(double* __restrict__ out, const double* __restrict__ tab,
                                              const B0Box* __restrict__ bx, const long* __restrict__ blk_off,
                                              int n_boxes) {
  extern __shared__ __align__(16) unsigned char fill_smem[];
  const long blk = blockIdx.x;
  int lo = 0, hi = n_boxes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (blk_off[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  const B0Box b = bx[lo];
  const int ni = b.ni, nj = b.nj, n_sd = b.n_sd;
  const long n2 = 2L * n_sd;
  const int nx2 = 2 * ni - 1, ny2 = 2 * nj - 1;
  const long per = (long)nx2 * ny2;
  long r = blk - blk_off[lo];
  const int jb = (int)(r % nj);
  r /= nj;
  const int ja = (int)(r % nj);
  r /= nj;
  const int cb = (int)(r & 1), ca = (int)(r >> 1);
  double* U = reinterpret_cast<double*>(fill_smem);
  double* V = U + nx2;
  const double* t = tab + b.tab_off + (long)((ca * 2 + cb) * 4) * per;
  const long r1 = (long)(ja - jb + nj - 1) * nx2, r2 = (long)(ja + jb) * nx2;
  for (int d = threadIdx.x; d < nx2; d += blockDim.x) {
    U[d] = t[r1 + d] - t[2 * per + r2 + d];
    V[d] = t[per + r1 + d] - t[3 * per + r2 + d];
  }
  __syncthreads();
  double* o = out + b.out_off + ((long)ca * n_sd + (long)ja * ni) * n2 + (long)cb * n_sd + (long)jb * ni;
  for (int e = threadIdx.x; e < ni * ni; e += blockDim.x) {
    const int ia = e / ni, ib = e - ia * ni;
    o[(long)ia * n2 + ib] = U[ia - ib + ni - 1] - V[ia + ib];
  }
}

// Dense B0 of a union of boxes (reading R16) from the stencil tables of its bounding box bx: one CTA per row
// (ca, pa) over all 2 n_sd columns, entries in the rounding order of k_fill, cross-box blocks included.
__global__ void __launch_bounds__(256) k_fill_union(double* __restrict__ out, const double* __restrict__ tab, B0Box bx,
                                                    int n_sd, const int* __restrict__ vert) {
  const int ni = bx.ni, nj = bx.nj, nx2 = 2 * ni - 1;
  const long per = (long)nx2 * (2 * nj - 1), n2 = 2L * n_sd;
  const long row = blockIdx.x;
  const int ca = row >= n_sd, pa = (int)(row - (long)ca * n_sd);
  const int ia = vert[2 * pa], ja = vert[2 * pa + 1];
  for (long col = threadIdx.x; col < n2; col += blockDim.x) {
    const int cb = col >= n_sd, pb = (int)(col - (long)cb * n_sd);
    out[row * n2 + col] = b0_entry(tab, per, nx2, ni, nj, ca, ja, ia, cb, vert[2 * pb + 1], vert[2 * pb]);
  }
}

}  // namespace

// The 16 stencil tables of every box (layout of k_tables) into a new device array *tab_out (caller frees
// it with cudaFree), tab_off of each box set; boxes must have their layout (b0_layout) filled in.
fsi_status b0_green_tables(fsi_ctx* c, std::vector<B0Box>& boxes, double** tab_out) {
  const int Nx = c->Nx, Mx = c->Mx, My = c->My;
  const double h = c->g.h;
  const int nb = (int)boxes.size();
  *tab_out = nullptr;
  long tab_n = 0, max_tab = 0;
  for (B0Box& b : boxes) {
    const long t = 16L * (2 * b.ni - 1) * (2 * b.nj - 1);
    b.tab_off = tab_n;
    tab_n += t;
    if (t > max_tab) max_tab = t;
  }
  std::vector<double> twx(4 * (size_t)Mx), twy(4 * (size_t)My);  // stage order of dst::block_fft
  int logLx = 0, logLy = 0, r3x = 1, r3y = 1;
  dst::split_length(2 * Mx, &logLx, &r3x);
  dst::split_length(2 * My, &logLy, &r3y);
  for (int p = 0; p < 2 * Mx; ++p) {
    const int m = dst::twiddle_exponent(p, logLx, r3x);
    twx[2 * p] = std::cos(-M_PI * (double)m / (double)Mx);
    twx[2 * p + 1] = std::sin(-M_PI * (double)m / (double)Mx);
  }
  for (int p = 0; p < 2 * My; ++p) {
    const int m = dst::twiddle_exponent(p, logLy, r3y);
    twy[2 * p] = std::cos(-M_PI * (double)m / (double)My);
    twy[2 * p + 1] = std::sin(-M_PI * (double)m / (double)My);
  }
  double *d_twx = nullptr, *d_twy = nullptr, *d_T1 = nullptr, *d_g = nullptr, *d_tab = nullptr;
  B0Box* d_bx = nullptr;
  fsi_status st = FSI_OK;
  do {
    if (ctx_dev_malloc(c, (void**)&d_twx, twx.size() * 8) != cudaSuccess || ctx_dev_malloc(c, (void**)&d_twy, twy.size() * 8) != cudaSuccess ||
        ctx_dev_malloc(c, (void**)&d_T1, (size_t)Nx * (My + 1) * 8) != cudaSuccess ||
        ctx_dev_malloc(c, (void**)&d_g, (size_t)(Mx + 1) * (My + 1) * 8) != cudaSuccess ||
        ctx_dev_malloc(c, (void**)&d_tab, (size_t)tab_n * 8) != cudaSuccess ||
        ctx_dev_malloc(c, (void**)&d_bx, (size_t)nb * sizeof(B0Box)) != cudaSuccess) {
      cudaGetLastError();
      st = FSI_ERR_OOM;
      break;
    }
    if (cudaMemcpyAsync(d_twx, twx.data(), twx.size() * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(d_twy, twy.data(), twy.size() * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(d_bx, boxes.data(), (size_t)nb * sizeof(B0Box), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess) {
      st = FSI_ERR_CUDA;
      break;
    }
    st = launch_dct1(nullptr, 0, 0, Nx, My, d_T1, My + 1, 1, (const double2*)d_twy, 2 * My, 1.0, c->lx,
                     c->ly, 1.0 / (h * h), 1.0 / c->g.dt, 0.5 / c->g.re, c->stream);
    if (st != FSI_OK) break;
    st = launch_dct1(d_T1, 1, My + 1, My + 1, Mx, d_g, 1, My + 1, (const double2*)d_twx, 2 * Mx,
                     1.0 / ((double)Mx * (double)My), nullptr, nullptr, 0.0, 0.0, 0.0, c->stream);
    if (st != FSI_OK) break;
    k_tables<<<dim3((unsigned)((max_tab + 127) / 128), nb), 128, 0, c->stream>>>(d_tab, d_bx, d_g, Mx, My, h);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) st = FSI_ERR_CUDA;
  } while (0);
  ctx_dev_free(c, d_twx);
  ctx_dev_free(c, d_twy);
  ctx_dev_free(c, d_T1);
  ctx_dev_free(c, d_g);
  ctx_dev_free(c, d_bx);
  if (st == FSI_OK) {
    *tab_out = d_tab;
  } else {
    ctx_dev_free(c, d_tab);
  }
  return st;
}

fsi_status b0_green(fsi_ctx* c, std::vector<B0Box>& boxes, double* out) {
  const int nb = (int)boxes.size();
  b0_layout(boxes);
  double* d_tab = nullptr;
  fsi_status st = b0_green_tables(c, boxes, &d_tab);
  if (st != FSI_OK) return st;
  B0Box* d_bx = nullptr;
  long* d_off = nullptr;
  do {
    std::vector<long> off(nb + 1, 0);
    int max_ni = 1;
    for (int k = 0; k < nb; ++k) {
      off[k + 1] = off[k] + 4L * boxes[k].nj * boxes[k].nj;
      if (boxes[k].ni > max_ni) max_ni = boxes[k].ni;
    }
    if (ctx_dev_malloc(c, (void**)&d_off, (size_t)(nb + 1) * sizeof(long)) != cudaSuccess ||
        ctx_dev_malloc(c, (void**)&d_bx, (size_t)nb * sizeof(B0Box)) != cudaSuccess) {
      cudaGetLastError();
      st = FSI_ERR_OOM;
      break;
    }
    if (cudaMemcpyAsync(d_off, off.data(), (size_t)(nb + 1) * sizeof(long), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_bx, boxes.data(), (size_t)nb * sizeof(B0Box), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess) {
      st = FSI_ERR_CUDA;
      break;
    }
    const size_t sm = (size_t)2 * (2 * max_ni - 1) * sizeof(double);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_fill<<<(unsigned)off[nb], 256, sm, c->stream>>>(out, d_tab, d_bx, d_off, nb);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) st = FSI_ERR_CUDA;
  } while (0);
  ctx_dev_free(c, d_tab);
  ctx_dev_free(c, d_bx);
  ctx_dev_free(c, d_off);
  return st;
}

fsi_status build_b0(fsi_ctx* c) {
  auto t0 = std::chrono::steady_clock::now();
  std::vector<B0Box> one(1, ctx_box(c));
  if (c->n_sdb > 1) {  // a union: tables of the bounding box, then every entry from its two points' vertices
    b0_layout(one);
    double* d_tab = nullptr;
    fsi_status st = b0_green_tables(c, one, &d_tab);
    if (st == FSI_OK) {
      k_fill_union<<<(unsigned)(2L * c->n_sd), 256, 0, c->stream>>>(c->B0, d_tab, one[0], c->n_sd, c->d_sd_vert);
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) st = FSI_ERR_CUDA;
    }
    ctx_dev_free(c, d_tab);
    c->b0_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
  }
  const fsi_status st = b0_green(c, one, c->B0);
  c->b0_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st;
}
