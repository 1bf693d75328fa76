// fsi_op_beam_solve: the structural linearisation and J_d solve of the FSI kernel (beam.cuh), run once on
// its own for testing.  One CTA of 128 threads; the flag's arrays live in shared memory as in the kernel.
#include <vector>
#include "beam.cuh"
#include "internal.h"

namespace {

struct OpArgs {
  beam::Flag F;  // ref points to global memory; the rest is set in the kernel
  const double *chi_n, *zeta_n, *zdot_n;
  const double* chi;
  const double* b;
  double* rz_out;
  double* x_out;
};

__global__ void __launch_bounds__(128) k_beam_op(OpArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = a.F.N, nd = 3 * N, t = threadIdx.x;
  double* chi = reinterpret_cast<double*>(sm);
  double* rz = chi + nd;
  double* cn = rz + nd;
  double* fab = cn + nd;
  float* ey = reinterpret_cast<float*>(fab + 6 * N);
  float* mi = ey + 12 * N;
  float* bm = mi + 6 * N;
  float* y = bm + 9 * N;
  beam::Flag F = a.F;
  F.chi = chi;
  F.fab = fab;
  F.ey = ey;
  F.mi = mi;
  F.bm = bm;
  F.rz = rz;
  F.y0 = nullptr;
  F.cn = cn;
  for (int g = t; g < nd; g += 128) {
    chi[g] = a.chi[g];
    cn[g] = beam::node_mass(F.mu, F.ds, N, g / 3, g % 3) *
            (F.four_dt2 * a.chi_n[g] + F.four_dt * a.zeta_n[g] + a.zdot_n[g]);
  }
  __syncthreads();
  beam::flag_elements(F, t, 128);
  __syncthreads();
  beam::flag_assemble(F, t, 128);
  for (int g = t; g < nd; g += 128) y[g] = (float)a.b[g];
  __syncthreads();
  const beam::Bcr B = beam::flag_bcr(F);
  beam::bcr_factor(B, t, 128, []() { __syncthreads(); });
  beam::bcr_solve(B, y, nd, 1, t, 128, []() { __syncthreads(); });
  for (int g = t; g < nd; g += 128) {
    a.rz_out[g] = rz[g];
    a.x_out[g] = (double)y[g];
  }
}

}  // namespace

extern "C" fsi_status fsi_op_beam_solve(int n_el, double ds, double mu, double ei, double ea, double cx, double cy,
                                        double dt, const double* chi, const double* chi_n, const double* zeta_n,
                                        const double* zetadot_n, const double* ref, const double* b, double* r_zeta,
                                        double* x) {
  if (n_el < 1 || n_el > 1000 || !(ds > 0) || !(mu > 0) || !(ei > 0) || !(ea > 0) || !(dt > 0) || !chi || !chi_n ||
      !zeta_n || !zetadot_n || !ref || !b)
    return FSI_ERR_INVALID_ARG;
  const size_t nd = 3 * (size_t)n_el;
  // device copies: chi, chi_n, zeta_n, zetadot_n, ref, b, then the outputs r_zeta, x
  std::vector<double> h(6 * nd);
  for (size_t k = 0; k < nd; ++k) {
    h[k] = chi[k];
    h[nd + k] = chi_n[k];
    h[2 * nd + k] = zeta_n[k];
    h[3 * nd + k] = zetadot_n[k];
    h[4 * nd + k] = ref[k];
    h[5 * nd + k] = b[k];
  }
  double* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 8 * nd * sizeof(double));
  if (e != cudaSuccess) {
    fsi_set_last_cuda_error(e, "fsi_op_beam_solve: cudaMalloc", __FILE__, __LINE__);
    return FSI_ERR_OOM;
  }
  const size_t smem = nd * 8 * 3 + (size_t)n_el * (6 * 8 + (12 + 6 + 9) * 4) + nd * 4;
  OpArgs a;
  a.F = beam::Flag{n_el,
                   cx,
                   cy,
                   mu,
                   ds,
                   beam::ElemParams{ds, ea / ds, 2.0 * ei / ds},
                   4.0 / (dt * dt),
                   4.0 / dt,
                   nullptr,
                   d + 4 * nd,
                   nullptr,
                   nullptr,
                   nullptr,
                   nullptr,
                   nullptr,
                   nullptr,
                   nullptr,
                   nullptr,
                   0};
  a.chi_n = d + nd;
  a.zeta_n = d + 2 * nd;
  a.zdot_n = d + 3 * nd;
  a.chi = d;
  a.b = d + 5 * nd;
  a.rz_out = d + 6 * nd;
  a.x_out = d + 7 * nd;
  fsi_status st = FSI_OK;
  e = cudaMemcpy(d, h.data(), 6 * nd * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_beam_op, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    k_beam_op<<<1, 128, smem>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  std::vector<double> out(2 * nd);
  if (e == cudaSuccess) e = cudaMemcpy(out.data(), d + 6 * nd, 2 * nd * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    fsi_set_last_cuda_error(e, "fsi_op_beam_solve", __FILE__, __LINE__);
    st = FSI_ERR_CUDA;
  } else {
    for (size_t k = 0; k < nd; ++k) {
      if (r_zeta) r_zeta[k] = out[k];
      if (x) x[k] = out[nd + k];
    }
  }
  cudaFree(d);
  return st;
}
