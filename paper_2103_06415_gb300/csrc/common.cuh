// Shared device/host helpers for the sub-domain IB-FSI library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/ibfsi.h"


// ---------------------------------------------------------------------------------------------
// Float pair: a value held as the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, 8 bytes like
// a double (the level fields of the mixed mode).  Sums and differences use Knuth's error-free two-sum and
// Dekker's fast two-sum (renormalisation) in float arithmetic only, so the difference of two nearby field
// values is exact up to the final rounding of the difference itself, without FP64 instructions or
// double-to-float conversions, both of which run at a small fraction of the FP32 rate on this GPU.
struct __align__(8) f2s {
  float hi, lo;
  f2s() = default;
  __host__ __device__ __forceinline__ f2s(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ explicit f2s(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ __forceinline__ explicit f2s(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ __forceinline__ explicit operator float() const { return hi + lo; }
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth's two-sum)
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// renormalise s + e with |e| small against |s| (Dekker's fast two-sum)
__host__ __device__ __forceinline__ f2s f2s_norm(float s, float e) {
  const float h = s + e;
  return f2s(h, e - (h - s));
}
__host__ __device__ __forceinline__ f2s operator+(f2s a, f2s b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return f2s_norm(s, e + (a.lo + b.lo));
}
__host__ __device__ __forceinline__ f2s operator-(f2s a, f2s b) {
  float s, e;
  two_sum(a.hi, -b.hi, s, e);
  return f2s_norm(s, e + (a.lo - b.lo));
}
// a * m for a float m: the product of hi exactly (fused multiply-add residual), the low part rounded
__host__ __device__ __forceinline__ f2s f2s_scale(f2s a, float m) {
  const float p = a.hi * m;
  const float e = fmaf(a.hi, m, -p);
  return f2s_norm(p, e + a.lo * m);
}
__host__ __device__ __forceinline__ f2s f2s_from_double(double v) {
  const float h = (float)v;
  return f2s(h, (float)(v - (double)h));
}

// Midpoint of two field values (ring values of a nested level)
template <typename T>
__host__ __device__ __forceinline__ T field_mid(T a, T b) { return T(0.5) * (a + b); }
template <>
__host__ __device__ __forceinline__ f2s field_mid<f2s>(f2s a, f2s b) {
  const f2s s = a + b;
  return f2s(0.5f * s.hi, 0.5f * s.lo);
}

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

#define FSI_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) {                                 \
      fsi_set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return FSI_ERR_CUDA;                                   \
    }                                                        \
  } while (0)

void fsi_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void fsi_set_last_message(const char* msg);

// First error wins: a kernel records a status code without trapping.
__device__ __forceinline__ void dev_set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Programmatic dependent launch: a kernel launched with pdl_launch may be set up by the GPU before its
// predecessor in the stream has finished; it waits (griddepcontrol.wait) until that predecessor has
// completed and its writes are visible.  Launched without the attribute, the wait is a no-op.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Raise, never lower, a kernel's dynamic shared-memory limit to `bytes`.  The limit belongs to the kernel for
// the whole process, and contexts of different sizes launch the same kernels: lowering it for a small
// context would make a larger one's next launch fail.
template <typename K>
inline cudaError_t raise_smem_limit(K kernel, size_t bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Row stride (in elements) for a vertex array of nx+1 columns, padded so rows start 32-byte aligned
// for both float and double.
static inline long padded_stride(int ncols) { return ((long)ncols + 7) / 8 * 8; }

static inline int ilog2_exact(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return ((1 << l) == v) ? l : -1;
}
