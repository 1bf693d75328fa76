// Allocation-free variant of the single-level DST solve (fsi_op_level_solve_noalloc, include/ibfsi_ops.h).
//
// Callers that cannot call cudaMalloc -- code running inside a framework whose allocator owns all device
// memory, or a hook that may not allocate on its path -- pass device inputs and outputs; the transform
// scratch (two transposed half-transforms and the sine/cosine tables) lives in the file-scope array
// g_noalloc_scratch below.  Every device that loads this library holds that array until the process exits.
//
// Host code must not use the array's name as a device address: it is a host-side stand-in.  The device
// address is taken once per device, with that device current, by cudaGetSymbolAddress on the first call
// made on the device (that first call should therefore come before any stream capture).  All calls share
// the array, and each call overwrites every scratch entry it later reads (nothing has to start at zero);
// calls whose work overlaps on the GPU race on the array and must be ordered by the caller.
#include <cmath>
#include <cstdio>
#include <mutex>
#include "dst.cuh"
#include "internal.h"
#include "../../include/ibfsi_ops.h"

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Tables for one call: twiddles exp(-2 pi i m / L) for both lengths (stage order of dst::block_fft) and
// lambda_k = 4 sin^2(pi k / 2M).
template <typename T>
__global__ void k_noalloc_tables(typename C2<T>::t* twx, int Lx, int logLx, typename C2<T>::t* twy, int Ly,
                                 int logLy, T* lx, int Mx, T* ly, int My) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < Lx) {
    double s, c;
    sincospi(-2.0 * (double)dst::twiddle_exponent(t, logLx) / (double)Lx, &s, &c);
    twx[t].x = (T)c;
    twx[t].y = (T)s;
  }
  if (t < Ly) {
    double s, c;
    sincospi(-2.0 * (double)dst::twiddle_exponent(t, logLy) / (double)Ly, &s, &c);
    twy[t].x = (T)c;
    twy[t].y = (T)s;
  }
  if (t <= Mx) {
    const double s = sinpi((double)t / (2.0 * Mx));
    lx[t] = T(4.0 * s * s);
  }
  if (t <= My) {
    const double s = sinpi((double)t / (2.0 * My));
    ly[t] = T(4.0 * s * s);
  }
}

struct Shape {
  int nthr, per, nf;
};
Shape shape_for(int logL) {  // same launch shapes as the context path: 4 * PER * threads = nf * L
  const int L = 1 << logL;
  Shape c;
  c.nthr = L / 4;
  if (c.nthr < 32) c.nthr = 32;
  if (c.nthr > 256) c.nthr = 256;
  c.per = 1;
  while (4 * c.per * c.nthr < L) c.per *= 2;
  c.nf = 4 * c.per * c.nthr / L;
  return c;
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
}

// Device address of the scratch array on the current device (set-up on first use per device).
fsi_status scratch_address(unsigned char** out) {
  int dev = -1;
  FSI_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FSI_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    FSI_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    set_attrs<float>();
    set_attrs<double>();
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_dev[dev];
  return FSI_OK;
}

template <typename T>
fsi_status solve_t(int nx, int ny, double h, double re, double dt, const T* rhs, T* w, T* s, cudaStream_t st) {
  using c2 = typename C2<T>::t;
  const int Nx = nx - 1, Ny = ny - 1, Mx = nx, My = ny;
  const int logLx = ilog2_exact(2 * nx), logLy = ilog2_exact(2 * ny);
  const int Lx = 1 << logLx, Ly = 1 << logLy;
  const long ldT = padded_stride(Ny), ldX = padded_stride(Nx);
  // scratch layout: T1 [Nx][ldT] | T2w [Ny][ldX] | T2s [Ny][ldX] | twx [Lx] | twy [Ly] | lx [Mx+1] | ly [My+1]
  size_t off[8];
  off[0] = 0;
  off[1] = off[0] + align256((size_t)Nx * ldT * sizeof(T));
  off[2] = off[1] + align256((size_t)Ny * ldX * sizeof(T));
  off[3] = off[2] + align256((size_t)Ny * ldX * sizeof(T));
  off[4] = off[3] + align256((size_t)Lx * sizeof(c2));
  off[5] = off[4] + align256((size_t)Ly * sizeof(c2));
  off[6] = off[5] + align256((size_t)(Mx + 1) * sizeof(T));
  off[7] = off[6] + align256((size_t)(My + 1) * sizeof(T));
  if (off[7] > kScratchBytes) {
    char msg[160];
    snprintf(msg, sizeof(msg), "fsi_op_level_solve_noalloc: %dx%d needs %zu bytes of scratch, limit %zu", nx, ny,
             off[7], kScratchBytes);
    fsi_set_last_message(msg);
    return FSI_ERR_UNSUPPORTED;
  }
  unsigned char* base = nullptr;
  fsi_status stt = scratch_address(&base);
  if (stt != FSI_OK) return stt;
  T* T1 = reinterpret_cast<T*>(base + off[0]);
  T* T2w = reinterpret_cast<T*>(base + off[1]);
  T* T2s = reinterpret_cast<T*>(base + off[2]);
  c2* twx = reinterpret_cast<c2*>(base + off[3]);
  c2* twy = reinterpret_cast<c2*>(base + off[4]);
  T* lx = reinterpret_cast<T*>(base + off[5]);
  T* ly = reinterpret_cast<T*>(base + off[6]);
  const int nt = (Lx > Ly ? Lx : Ly) + 1;
  k_noalloc_tables<T><<<(nt + 255) / 256, 256, 0, st>>>(twx, Lx, logLx, twy, Ly, logLy, lx, Mx, ly, My);
  const Shape cx = shape_for(logLx), cy = shape_for(logLy);
  {  // forward x, transposed into T1
    dim3 grid((Ny + 2 * cx.nf - 1) / (2 * cx.nf));
    const size_t sm = dst::pass_smem<T>((size_t)cx.nf * Lx, Lx);
    if (cx.per == 1) dst::k_xf<T, 1><<<grid, cx.nthr, sm, st>>>(rhs, Nx, 0, Ny, Nx, T1, ldT, 0, twx, logLx, cx.nf);
    else if (cx.per == 2) dst::k_xf<T, 2><<<grid, cx.nthr, sm, st>>>(rhs, Nx, 0, Ny, Nx, T1, ldT, 0, twx, logLx, cx.nf);
    else dst::k_xf<T, 4><<<grid, cx.nthr, sm, st>>>(rhs, Nx, 0, Ny, Nx, T1, ldT, 0, twx, logLx, cx.nf);
  }
  {  // y: forward, diagonal A_w^{-1} and Lap^{-1}, inverse; zero boundary values (no ring terms)
    dst::SpecParams<T> sp = {};
    sp.lx = lx;
    sp.ly = ly;
    sp.ring = nullptr;
    sp.inv_h2 = T(1.0 / (h * h));
    sp.inv_dt = T(1.0 / dt);
    sp.inv_2re = T(0.5 / re);
    sp.norm = T(4.0 / ((double)Mx * (double)My));
    sp.ring_w = T(0);
    sp.Mx = Mx;
    sp.My = My;
    dim3 grid((Nx + 2 * cy.nf - 1) / (2 * cy.nf));
    const size_t sm = dst::pass_smem<T>((size_t)2 * cy.nf * Ly, Ly);
    if (cy.per == 1) dst::k_ysolve<T, 1><<<grid, cy.nthr, sm, st>>>(T1, ldT, 0, Nx, Ny, T2w, T2s, ldX, 0, twy, logLy, cy.nf, sp, (const T*)nullptr);
    else if (cy.per == 2) dst::k_ysolve<T, 2><<<grid, cy.nthr, sm, st>>>(T1, ldT, 0, Nx, Ny, T2w, T2s, ldX, 0, twy, logLy, cy.nf, sp, (const T*)nullptr);
    else dst::k_ysolve<T, 4><<<grid, cy.nthr, sm, st>>>(T1, ldT, 0, Nx, Ny, T2w, T2s, ldX, 0, twy, logLy, cy.nf, sp, (const T*)nullptr);
  }
  {  // inverse x into the interior of the caller's vertex arrays (row stride nx + 1)
    dim3 grid(dst::xi_blocks(Ny, cx.nf));
    const size_t sm = dst::pass_smem<T>((size_t)cx.nf * Lx, Lx);
    const long fld = nx + 1;
    if (cx.per == 1) dst::k_xi<T, 1><<<grid, cx.nthr, sm, st>>>(T2w, T2s, ldX, 0, Ny, Nx, w, s, fld, 0, 0, twx, logLx, cx.nf);
    else if (cx.per == 2) dst::k_xi<T, 2><<<grid, cx.nthr, sm, st>>>(T2w, T2s, ldX, 0, Ny, Nx, w, s, fld, 0, 0, twx, logLx, cx.nf);
    else dst::k_xi<T, 4><<<grid, cx.nthr, sm, st>>>(T2w, T2s, ldX, 0, Ny, Nx, w, s, fld, 0, 0, twx, logLx, cx.nf);
  }
  FSI_CUDA_TRY(cudaGetLastError());
  return FSI_OK;
}

}  // namespace

extern "C" fsi_status fsi_op_level_solve_noalloc(int precision, int nx, int ny, double h, double re, double dt,
                                                 const void* rhs_dev, void* w_dev, void* s_dev, void* stream) {
  if (!rhs_dev || !w_dev || !s_dev) return FSI_ERR_INVALID_ARG;
  const bool pow2 = nx >= 16 && ny >= 16 && (nx & (nx - 1)) == 0 && (ny & (ny - 1)) == 0 && nx <= 2048 &&
                    ny <= 2048;
  if (!pow2 || !(h > 0) || !(re > 0) || !(dt > 0)) return FSI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == FSI_PREC_FP64)
    return solve_t<double>(nx, ny, h, re, dt, (const double*)rhs_dev, (double*)w_dev, (double*)s_dev, st);
  if (precision == FSI_PREC_FP32)
    return solve_t<float>(nx, ny, h, re, dt, (const float*)rhs_dev, (float*)w_dev, (float*)s_dev, st);
  return FSI_ERR_INVALID_ARG;
}
