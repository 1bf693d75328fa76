// Saving and loading the precomputed sub-domain operator.  B0 (or the filtered B0' of Eq. filtereq) depends
// only on the finest grid (cell counts and spacing), the time step, the Reynolds number and Omega_0, not on
// the bodies, so one build serves every run that shares them -- e.g. a parametric study over body stiffness
// or mass (the reuse noted after Algorithm 1).
//
// File: a fixed header (below), then the operator as doubles in the context's device layout: the dense
// (2 n_sd)^2 row-major B0, or the windowed columns of B0' ([2 n_sd][2][2w+1][2w+1]).  Native byte order.
#include <cstdio>
#include <cstring>
#include <vector>
#include "internal.h"

namespace {

struct OpHeader {
  char magic[8];  // "IBFSIB0"
  int32_t version, format;  // format 0: dense B0, 1: windowed B0'
  int32_t nx, ny, i_lo, i_hi, j_lo, j_hi, window, pad;
  double h, re, dt, drop_tol;
  int64_t values, nnz;
};

constexpr char kMagic[8] = {'I', 'B', 'F', 'S', 'I', 'B', '0', '\0'};
constexpr size_t kChunk = (size_t)8 << 20;  // doubles per staged copy (64 MB)

OpHeader header_of(const fsi_ctx* c) {
  OpHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kMagic, 8);
  hd.version = 1;
  hd.format = c->Bw ? 1 : 0;
  hd.nx = c->nx;
  hd.ny = c->ny;
  hd.i_lo = c->i_lo;
  hd.i_hi = c->i_hi;
  hd.j_lo = c->j_lo;
  hd.j_hi = c->j_hi;
  hd.window = c->Bw ? c->bw : 0;
  hd.h = c->g.h;
  hd.re = c->g.re;
  hd.dt = c->g.dt;
  hd.drop_tol = c->drop_tol;
  const long n2 = 2L * c->n_sd, side = 2L * hd.window + 1;
  hd.values = c->Bw ? n2 * 2 * side * side : n2 * n2;
  hd.nnz = c->Bw ? c->b0_nnz : n2 * n2;
  return hd;
}

}  // namespace

extern "C" fsi_status fsi_save_operator(fsi_ctx* c, const char* path) {
  if (!c || !path) return FSI_ERR_INVALID_ARG;
  if (!c->have_b0) return FSI_ERR_STATE;
  if (!c->B0 && !c->Bw) return FSI_ERR_UNSUPPORTED;  // true-E coupling: no operator
  if (c->n_app > 0) return FSI_ERR_UNSUPPORTED;        // appended points are not recorded in the header
  if (c->n_sdb > 1) return FSI_ERR_UNSUPPORTED;        // nor are the boxes of a union
  const OpHeader hd = header_of(c);
  const double* src = c->Bw ? c->Bw : c->B0;
  FILE* f = fopen(path, "wb");
  if (!f) {
    fsi_set_last_message("fsi_save_operator: cannot open the file for writing");
    return FSI_ERR_INVALID_ARG;
  }
  fsi_status st = FSI_OK;
  if (fwrite(&hd, sizeof(hd), 1, f) != 1) st = FSI_ERR_INVALID_ARG;
  std::vector<double> buf;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) st = FSI_ERR_CUDA;
  for (int64_t o = 0; st == FSI_OK && o < hd.values; o += (int64_t)kChunk) {
    const size_t n = (size_t)std::min<int64_t>((int64_t)kChunk, hd.values - o);
    buf.resize(n);
    if (cudaMemcpy(buf.data(), src + o, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) st = FSI_ERR_CUDA;
    else if (fwrite(buf.data(), 8, n, f) != n) st = FSI_ERR_INVALID_ARG;
  }
  if (fclose(f) != 0 && st == FSI_OK) st = FSI_ERR_INVALID_ARG;
  if (st == FSI_ERR_INVALID_ARG) fsi_set_last_message("fsi_save_operator: short write");
  if (st == FSI_ERR_CUDA) cudaGetLastError();
  return st;
}

// Reads the operator for fsi_load_operator (after the context's checks): the header must match this
// context's grid, Omega_0, time step and Reynolds number exactly.
fsi_status load_operator_data(fsi_ctx* c, const char* path) {
  FILE* f = fopen(path, "rb");
  if (!f) {
    fsi_set_last_message("fsi_load_operator: cannot open the file");
    return FSI_ERR_INVALID_ARG;
  }
  OpHeader hd;
  fsi_status st = FSI_OK;
  if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, kMagic, 8) != 0 || hd.version != 1 ||
      (hd.format != 0 && hd.format != 1)) {
    fsi_set_last_message("fsi_load_operator: not an operator file of this library");
    st = FSI_ERR_INVALID_ARG;
  } else if (hd.nx != c->nx || hd.ny != c->ny || hd.i_lo != c->i_lo || hd.i_hi != c->i_hi || hd.j_lo != c->j_lo ||
             hd.j_hi != c->j_hi || hd.h != c->g.h || hd.re != c->g.re || hd.dt != c->g.dt) {
    fsi_set_last_message("fsi_load_operator: grid, Omega_0, Re or dt differ from the file's");
    st = FSI_ERR_INVALID_ARG;
  }
  const long n2 = 2L * c->n_sd, side = 2L * hd.window + 1;
  if (st == FSI_OK) {
    const int64_t expect = hd.format == 1 ? n2 * 2 * side * side : n2 * n2;
    if (hd.values != expect || (hd.format == 1 && hd.window < 1)) {
      fsi_set_last_message("fsi_load_operator: operator size does not match Omega_0");
      st = FSI_ERR_INVALID_ARG;
    }
  }
  double* dst = nullptr;
  if (st == FSI_OK && !(dst = (double*)ctx_alloc(c, (size_t)hd.values * 8))) st = FSI_ERR_OOM;
  std::vector<double> buf;
  for (int64_t o = 0; st == FSI_OK && o < hd.values; o += (int64_t)kChunk) {
    const size_t n = (size_t)std::min<int64_t>((int64_t)kChunk, hd.values - o);
    buf.resize(n);
    if (fread(buf.data(), 8, n, f) != n) {
      fsi_set_last_message("fsi_load_operator: short read");
      st = FSI_ERR_INVALID_ARG;
    } else if (cudaMemcpy(dst + o, buf.data(), n * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      st = FSI_ERR_CUDA;
    }
  }
  fclose(f);
  if (st != FSI_OK) return st;
  if (hd.format == 1) {
    c->Bw = dst;
    c->bw = hd.window;
    c->b0_nnz = hd.nnz;
  } else {
    c->B0 = dst;
  }
  c->drop_tol = hd.drop_tol;
  return FSI_OK;
}
