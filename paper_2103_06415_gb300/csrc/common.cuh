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

// Row stride (in elements) for a vertex array of nx+1 columns, padded so rows start 32-byte aligned
// for both float and double.
static inline long padded_stride(int ncols) { return ((long)ncols + 7) / 8 * 8; }

static inline int ilog2_exact(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return ((1 << l) == v) ? l : -1;
}
