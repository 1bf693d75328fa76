// Checkpoint and resume of a run: everything the next step reads, so that n steps, a save, a load into a
// context set up the same way and n more steps reproduce 2n uninterrupted steps bit for bit.
//
// Saved: the vorticity, streamfunction and previous advection term of every level; per body the structural
// state; the last surface stress f (the flags' warm start); the deformable state (chi, zeta, zetadot and the
// reference chords); the float inverse of the small system (both ping-pong buffers) with the control words
// that say which is current and valid; the interpolation map of the last step; the history ring; the step
// counters; the true-E loop counters.  The file starts with a header that fixes the context's shape.
#include <cstdio>
#include <cstring>
#include <vector>
#include "internal.h"

int fsi_float_ld(int nf);

namespace {

struct StateHeader {
  char magic[8];  // "IBFSIST"
  int32_t version, precision;
  int32_t nx, ny, n_levels, nb, nf, n_bodies, nd_tot, ne_tot, hist_cap, coupling;
  double h, re, dt;
  int64_t steps_done;
  int32_t first_pending, n_blobs;
};

constexpr char kMagic[8] = {'I', 'B', 'F', 'S', 'I', 'S', 'T', '\0'};

struct Blob {
  void* dev;
  size_t bytes;
};

// the device buffers of the state, in file order (absent ones have zero size)
std::vector<Blob> blobs(fsi_ctx* c) {
  const size_t lvl = (size_t)c->G * c->lvl_elems * c->fesz;
  const size_t xbytes = c->nf > 0 ? (size_t)c->nf * fsi_float_ld(c->nf) * 4 : 0;
  std::vector<Blob> b = {
      {c->w_all, lvl},
      {c->s_all, lvl},
      {c->nprev_all, lvl},
      {c->d_state, c->d_state ? (size_t)c->n_bodies * sizeof(BodyState) : 0},
      {c->d_f, c->d_f ? (size_t)c->nf * 8 : 0},
      {c->d_ctrl, 64},
      {c->d_Kinv, c->d_Kinv ? xbytes : 0},
      {c->d_W, c->d_W ? xbytes : 0},
      {c->d_pidx, c->d_pidx ? (size_t)c->nb * 4 * sizeof(int) : 0},
      {c->d_pw, c->d_pw ? (size_t)c->nb * 4 * 8 : 0},
      {c->d_pcij, c->d_pcij ? (size_t)c->nb * 2 * sizeof(int) : 0},
      {c->d_hist, c->d_hist ? (size_t)c->hist_cap * c->n_bodies * 6 * 8 : 0},
      {c->d_bchi, c->d_bchi ? (size_t)c->nd_tot * 8 : 0},
      {c->d_bzeta, c->d_bzeta ? (size_t)c->nd_tot * 8 : 0},
      {c->d_bzdot, c->d_bzdot ? (size_t)c->nd_tot * 8 : 0},
      {c->d_bref, c->d_bref ? (size_t)c->nd_tot * 8 : 0},
      {c->d_te_ctl, c->d_te_ctl ? 16 * sizeof(int) : 0},
      {c->d_te_total, c->d_te_total ? sizeof(unsigned long long) : 0},
  };
  return b;
}

StateHeader header_of(const fsi_ctx* c, int n_blobs) {
  StateHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kMagic, 8);
  hd.version = 1;
  hd.precision = c->prec;
  hd.nx = c->nx;
  hd.ny = c->ny;
  hd.n_levels = c->G;
  hd.nb = c->nb;
  hd.nf = c->nf;
  hd.n_bodies = c->n_bodies;
  hd.nd_tot = c->nd_tot;
  hd.ne_tot = c->ne_tot;
  hd.hist_cap = c->hist_cap;
  hd.coupling = c->x.coupling;
  hd.h = c->g.h;
  hd.re = c->g.re;
  hd.dt = c->g.dt;
  hd.steps_done = c->steps_done;
  hd.first_pending = c->first_pending;
  hd.n_blobs = n_blobs;
  return hd;
}

}  // namespace

extern "C" fsi_status fsi_save_state(fsi_ctx* c, const char* path) {
  if (!c || !path) return FSI_ERR_INVALID_ARG;
  NvtxRange range("fsi_save_state");
  if (c->nb > 0 && c->stage < 1) return FSI_ERR_STATE;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  const std::vector<Blob> bl = blobs(c);
  const StateHeader hd = header_of(c, (int)bl.size());
  FILE* f = fopen(path, "wb");
  if (!f) {
    fsi_set_last_message("fsi_save_state: cannot open the file for writing");
    return FSI_ERR_INVALID_ARG;
  }
  fsi_status st = fwrite(&hd, sizeof(hd), 1, f) == 1 ? FSI_OK : FSI_ERR_INVALID_ARG;
  std::vector<char> buf;
  for (const Blob& b : bl) {
    if (st != FSI_OK) break;
    const uint64_t n = b.dev ? b.bytes : 0;
    if (fwrite(&n, sizeof(n), 1, f) != 1) {
      st = FSI_ERR_INVALID_ARG;
      break;
    }
    if (n == 0) continue;
    buf.resize(n);
    if (cudaMemcpy(buf.data(), b.dev, n, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      st = FSI_ERR_CUDA;
    } else if (fwrite(buf.data(), 1, n, f) != n) {
      st = FSI_ERR_INVALID_ARG;
    }
  }
  if (fclose(f) != 0 && st == FSI_OK) st = FSI_ERR_INVALID_ARG;
  if (st == FSI_ERR_INVALID_ARG) fsi_set_last_message("fsi_save_state: short write");
  return st;
}

extern "C" fsi_status fsi_load_state(fsi_ctx* c, const char* path) {
  if (!c || !path) return FSI_ERR_INVALID_ARG;
  NvtxRange range("fsi_load_state");
  if (c->nb > 0 && c->stage < 1) return FSI_ERR_STATE;
  FILE* f = fopen(path, "rb");
  if (!f) {
    fsi_set_last_message("fsi_load_state: cannot open the file");
    return FSI_ERR_INVALID_ARG;
  }
  const std::vector<Blob> bl = blobs(c);
  StateHeader hd, want = header_of(c, (int)bl.size());
  fsi_status st = FSI_OK;
  if (fread(&hd, sizeof(hd), 1, f) != 1 || memcmp(hd.magic, kMagic, 8) != 0 || hd.version != 1) {
    fsi_set_last_message("fsi_load_state: not a state file of this library");
    st = FSI_ERR_INVALID_ARG;
  } else if (hd.precision != want.precision || hd.nx != want.nx || hd.ny != want.ny || hd.n_levels != want.n_levels ||
             hd.nb != want.nb || hd.nf != want.nf || hd.n_bodies != want.n_bodies || hd.nd_tot != want.nd_tot ||
             hd.ne_tot != want.ne_tot || hd.hist_cap != want.hist_cap || hd.coupling != want.coupling ||
             hd.h != want.h || hd.re != want.re || hd.dt != want.dt || hd.n_blobs != want.n_blobs) {
    fsi_set_last_message("fsi_load_state: the file was written by a context of another shape");
    st = FSI_ERR_INVALID_ARG;
  }
  // read everything to the host first, so that a short or mismatched file leaves the context unchanged
  std::vector<std::vector<char>> data(bl.size());
  for (size_t k = 0; st == FSI_OK && k < bl.size(); ++k) {
    uint64_t n = 0;
    if (fread(&n, sizeof(n), 1, f) != 1 || n != (bl[k].dev ? bl[k].bytes : 0)) {
      fsi_set_last_message("fsi_load_state: truncated or mismatched state");
      st = FSI_ERR_INVALID_ARG;
      break;
    }
    data[k].resize(n);
    if (n > 0 && fread(data[k].data(), 1, n, f) != n) {
      fsi_set_last_message("fsi_load_state: truncated state");
      st = FSI_ERR_INVALID_ARG;
    }
  }
  fclose(f);
  if (st != FSI_OK) return st;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (size_t k = 0; k < bl.size(); ++k)
    if (!data[k].empty()) FSI_CUDA_TRY(cudaMemcpy(bl[k].dev, data[k].data(), data[k].size(), cudaMemcpyHostToDevice));
  c->steps_done = hd.steps_done;
  c->first_pending = hd.first_pending;
  return FSI_OK;
}
