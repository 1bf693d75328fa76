// Shared device/host helpers for the sub-domain IB-FSI library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/ibfsi.h"

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
