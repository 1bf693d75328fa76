// C ABI: context life cycle, offline/online stages and read-back (see include/ibfsi.h).
#include <cstddef>
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <new>
#include <vector>
#include "dst.cuh"
#include "internal.h"

int fsi_kernel_max_ctas_per_sm(const fsi_ctx* c);
size_t fsi_smem_bytes(const fsi_ctx* c);
bool fsi_smem_fits(const fsi_ctx* c, bool big);
double beam_initial_state(const BodyHost& h, double ds, double tip, double* chi, double* zeta, double* zdot,
                          double* ref);
int fsi_min_grid(int nf, bool big);
int fsi_float_ld(int nf);

static thread_local char g_errmsg[512] = "";

void fsi_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_errmsg, sizeof(g_errmsg), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

void fsi_set_last_message(const char* msg) { snprintf(g_errmsg, sizeof(g_errmsg), "%s", msg); }

extern "C" const char* fsi_last_error_message(void) { return g_errmsg; }

extern "C" const char* fsi_status_string(int s) {
  switch (s) {
    case FSI_OK: return "ok";
    case FSI_ERR_INVALID_ARG: return "invalid argument";
    case FSI_ERR_OOM: return "out of device memory";
    case FSI_ERR_UNSUPPORTED: return "unsupported";
    case FSI_ERR_BODY_OUTSIDE_SUBDOMAIN: return "body point outside the sub-domain";
    case FSI_ERR_NOT_CONVERGED: return "FSI iteration did not converge";
    case FSI_ERR_NONFINITE: return "non-finite value";
    case FSI_ERR_TIMEOUT: return "timeout";
    case FSI_ERR_CUDA: return "CUDA error";
    case FSI_ERR_STATE: return "call made in the wrong stage";
    default: return "unknown status";
  }
}

cudaError_t ctx_dev_malloc(const fsi_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (!c->x.dev_alloc) return cudaMalloc(p, bytes);
  void* q = c->x.dev_alloc(bytes, c->x.dev_alloc_user);
  if (q && (reinterpret_cast<uintptr_t>(q) & 255u) != 0) {  // TMA and vector loads need the alignment
    c->x.dev_free(q, c->x.dev_alloc_user);
    q = nullptr;
  }
  if (!q) return cudaErrorMemoryAllocation;
  *p = q;
  return cudaSuccess;
}

void ctx_dev_free(const fsi_ctx* c, void* p) {
  if (!p) return;
  if (c->x.dev_alloc)
    c->x.dev_free(p, c->x.dev_alloc_user);
  else
    cudaFree(p);
}

void* ctx_alloc(fsi_ctx* c, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx_dev_malloc(c, &p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaMemsetAsync(p, 0, bytes, c->stream);
  c->allocs.push_back(p);
  c->dev_bytes += bytes;
  return p;
}

static void ctx_free_all(fsi_ctx* c) {
  for (void* p : c->allocs) ctx_dev_free(c, p);
  c->allocs.clear();
  c->dev_bytes = 0;
}

// Cells per axis: 2^k or 3 * 2^k in [16, 2048] (the sine-transform length 2n is then 2^(k+1) or 3 * 2^(k+1)).
static bool cells_ok(int n) {
  int logP = 0, r3 = 1;
  return n >= 16 && n <= 2048 && dst::split_length(2 * n, &logP, &r3);
}

// The ring transforms of a grid with a 3 * 2^k axis run with one butterfly set per thread: both axes' lengths
// must then have power-of-two parts of at most 1024 (e.g. 1536 x 768, 1536 x 512, 768 x 512).
static bool grid_ok(int nx, int ny) {
  int lx = 0, ly = 0, rx = 1, ry = 1;
  if (!cells_ok(nx) || !cells_ok(ny)) return false;
  dst::split_length(2 * nx, &lx, &rx);
  dst::split_length(2 * ny, &ly, &ry);
  return (rx == 1 && ry == 1) || (lx <= 10 && ly <= 10);
}

// Complex twiddles of length L = r3 2^logP in the stage order of dst::block_fft (entry p: m =
// twiddle_exponent(p, logP, r3)).
template <typename T>
static fsi_status upload_twiddles(fsi_ctx* c, int L, void** out) {
  std::vector<T> tw(2 * (size_t)L);
  int logP = 0, r3 = 1;
  dst::split_length(L, &logP, &r3);
  for (int p = 0; p < L; ++p) {
    const int m = dst::twiddle_exponent(p, logP, r3);
    const double a = -2.0 * M_PI * (double)m / (double)L;
    tw[2 * p] = (T)std::cos(a);
    tw[2 * p + 1] = (T)std::sin(a);
  }
  *out = ctx_alloc(c, tw.size() * sizeof(T));
  if (!*out) return FSI_ERR_OOM;
  FSI_CUDA_TRY(cudaMemcpyAsync(*out, tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  return FSI_OK;
}

static fsi_status upload_d(fsi_ctx* c, const std::vector<double>& v, double** out) {
  *out = (double*)ctx_alloc(c, v.size() * 8);
  if (!*out) return FSI_ERR_OOM;
  FSI_CUDA_TRY(cudaMemcpyAsync(*out, v.data(), v.size() * 8, cudaMemcpyHostToDevice, c->stream));
  return FSI_OK;
}

static fsi_status upload_f(fsi_ctx* c, const std::vector<double>& v, void** out) {
  std::vector<float> f(v.begin(), v.end());
  *out = ctx_alloc(c, f.size() * 4);
  if (!*out) return FSI_ERR_OOM;
  FSI_CUDA_TRY(cudaMemcpyAsync(*out, f.data(), f.size() * 4, cudaMemcpyHostToDevice, c->stream));
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));  // f is a temporary
  return FSI_OK;
}

#define TRY(x)                       \
  do {                               \
    fsi_status _s = (x);             \
    if (_s != FSI_OK) return _s;     \
  } while (0)

static fsi_status create_impl(fsi_ctx* c) {
  const fsi_grid_desc& g = c->g;
  c->G = g.n_levels;
  c->nx = g.nx;
  c->ny = g.ny;
  c->Nx = g.nx - 1;
  c->Ny = g.ny - 1;
  c->Mx = g.nx;
  c->My = g.ny;
  dst::split_length(2 * g.nx, &c->logPx, &c->r3x);
  dst::split_length(2 * g.ny, &c->logPy, &c->r3y);
  c->ps = padded_stride(g.nx + 1);
  c->lvl_elems = (long)(g.ny + 1) * c->ps;
  c->ldT = padded_stride(c->Ny);
  c->ldX = padded_stride(c->Nx);
  c->ring_ld = padded_stride(c->Nx > c->Ny ? c->Nx : c->Ny);
  const size_t E = c->esz;
  // the mixed mode keeps a second right-hand-side slot (and x-transform slot) per level: the defect of the
  // level's streamfunction, transformed with the right-hand sides (fluid.cu)
  const int slots = c->prec == FSI_PREC_MIXED ? 2 * c->G : c->G;
  const size_t lvl = (size_t)slots * c->lvl_elems * E;
  const size_t flvl = (size_t)c->G * c->lvl_elems * c->fesz;
  if (!(c->w_all = ctx_alloc(c, flvl)) || !(c->s_all = ctx_alloc(c, flvl)) || !(c->nprev_all = ctx_alloc(c, flvl)) ||
      !(c->rhs_all = ctx_alloc(c, lvl)) || !(c->T1 = ctx_alloc(c, (size_t)slots * c->Nx * c->ldT * E)) ||
      !(c->T2w = ctx_alloc(c, (size_t)c->Ny * c->ldX * E)) || !(c->T2s = ctx_alloc(c, (size_t)c->Ny * c->ldX * E)) ||
      !(c->src = ctx_alloc(c, (size_t)c->lvl_elems * E)) || !(c->ring = ctx_alloc(c, (size_t)8 * c->ring_ld * E)))
    return FSI_ERR_OOM;
  std::vector<double> lx(c->Mx + 1), ly(c->My + 1), sx1(c->Mx + 1), sxN(c->Mx + 1), sy1(c->My + 1), syN(c->My + 1);
  for (int k = 0; k <= c->Mx; ++k) {
    const double s = std::sin(M_PI * k / (2.0 * c->Mx));
    lx[k] = 4.0 * s * s;
    sx1[k] = std::sin(M_PI * k / (double)c->Mx);
    sxN[k] = std::sin(M_PI * (double)k * c->Nx / (double)c->Mx);
  }
  for (int l = 0; l <= c->My; ++l) {
    const double s = std::sin(M_PI * l / (2.0 * c->My));
    ly[l] = 4.0 * s * s;
    sy1[l] = std::sin(M_PI * l / (double)c->My);
    syN[l] = std::sin(M_PI * (double)l * c->Ny / (double)c->My);
  }
  TRY(upload_d(c, lx, &c->lx));
  TRY(upload_d(c, ly, &c->ly));
  TRY(upload_d(c, sx1, &c->sx1));
  TRY(upload_d(c, sxN, &c->sxN));
  TRY(upload_d(c, sy1, &c->sy1));
  TRY(upload_d(c, syN, &c->syN));
  if (c->prec == FSI_PREC_FP64) {
    c->lxT = c->lx;
    c->lyT = c->ly;
    c->sx1T = c->sx1;
    c->sxNT = c->sxN;
    c->sy1T = c->sy1;
    c->syNT = c->syN;
  } else {
    TRY(upload_f(c, lx, &c->lxT));
    TRY(upload_f(c, ly, &c->lyT));
    TRY(upload_f(c, sx1, &c->sx1T));
    TRY(upload_f(c, sxN, &c->sxNT));
    TRY(upload_f(c, sy1, &c->sy1T));
    TRY(upload_f(c, syN, &c->syNT));
  }
  if (c->prec == FSI_PREC_FP64) {
    TRY(upload_twiddles<double>(c, 2 * c->Mx, &c->twx));
    TRY(upload_twiddles<double>(c, 2 * c->My, &c->twy));
  } else {
    TRY(upload_twiddles<float>(c, 2 * c->Mx, &c->twx));
    TRY(upload_twiddles<float>(c, 2 * c->My, &c->twy));
  }
  if (!(c->d_status = (int*)ctx_alloc(c, 64)) || !(c->d_ctrl = (int*)ctx_alloc(c, 64))) return FSI_ERR_OOM;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return FSI_OK;
}

// Time each sine-transform pass of a level solve (level 0, zero right-hand side, zero fields) with CUDA
// events around every launch of that pass; avg_us[p] for the current dst_gemm choice.
static fsi_status time_dst_passes(fsi_ctx* c, int reps, double* avg_us) {
  for (int k = 0; k < 3; ++k) TRY(launch_level_solve(c, 0, c->src, c->w_all, c->s_all, 0, 0));  // warm-up
  for (int p = 0; p < 3; ++p) {
    c->prof_ev.assign(2 * reps, nullptr);
    fsi_status st = FSI_OK;
    for (cudaEvent_t& e : c->prof_ev)
      if (cudaEventCreate(&e) != cudaSuccess) st = FSI_ERR_CUDA;
    c->prof_class = KC_XF + p;
    c->prof_used = 0;
    for (int r = 0; st == FSI_OK && r < reps; ++r) st = launch_level_solve(c, 0, c->src, c->w_all, c->s_all, 0, 0);
    c->prof_class = KC_NONE;
    if (st == FSI_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = FSI_ERR_CUDA;
    double sum = 0.0;
    int n = 0;
    for (int k = 0; st == FSI_OK && k + 1 < c->prof_used; k += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, c->prof_ev[k], c->prof_ev[k + 1]) != cudaSuccess) st = FSI_ERR_CUDA;
      sum += ms;
      ++n;
    }
    for (cudaEvent_t e : c->prof_ev)
      if (e) cudaEventDestroy(e);
    c->prof_ev.clear();
    c->prof_used = 0;
    if (st != FSI_OK) return st;
    avg_us[p] = n ? 1e3 * sum / n : 0.0;
  }
  return FSI_OK;
}

// Choose FFT or tensor-core GEMM for each sine-transform pass (fsi_exec_desc.dst_method).  Autotuned
// choices are cached per grid shape so every context of one process with that grid takes the same path.
static fsi_status dst_select(fsi_ctx* c) {
  const int m = c->x.dst_method;
  if (m == 0 || c->prec != FSI_PREC_FP32 || !gemm_dst_supported(c->nx, c->ny)) return FSI_OK;
  fsi_status st = gemm_dst_setup(c);
  if (st != FSI_OK) {
    gemm_dst_free(c);
    return m == 1 ? st : FSI_OK;  // autotune falls back to the FFT passes
  }
  if (m == 1) {
    c->dst_gemm[0] = c->dst_gemm[1] = c->dst_gemm[2] = 1;
    return FSI_OK;
  }
  static std::mutex mu;
  static std::map<std::pair<int, int>, std::array<double, 6>> cache;
  std::lock_guard<std::mutex> lock(mu);
  const std::pair<int, int> key(c->nx, c->ny);
  auto it = cache.find(key);
  std::array<double, 6> us{};
  if (it != cache.end()) {
    us = it->second;
  } else {
    for (int impl = 0; impl < 2; ++impl) {
      c->dst_gemm[0] = c->dst_gemm[1] = c->dst_gemm[2] = impl;
      TRY(time_dst_passes(c, 20, &us[3 * impl]));
    }
    int dev_status = 0;
    FSI_CUDA_TRY(cudaMemcpy(&dev_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (dev_status != 0) return (fsi_status)dev_status;
    cache[key] = us;
  }
  for (int p = 0; p < 3; ++p) {
    c->dst_us[0][p] = us[p];
    c->dst_us[1][p] = us[3 + p];
    c->dst_gemm[p] = us[3 + p] < us[p] ? 1 : 0;
  }
  c->launches_per_step = 0;
  return FSI_OK;
}

extern "C" fsi_status fsi_create(const fsi_grid_desc* grid, const fsi_exec_desc* exec, fsi_ctx** out) {
  if (!grid || !out) return FSI_ERR_INVALID_ARG;
  *out = nullptr;
  if (!grid_ok(grid->nx, grid->ny) || grid->n_levels < 1 || grid->n_levels > 12 || !(grid->h > 0) ||
      !(grid->re > 0) || !(grid->dt > 0) || !std::isfinite(grid->x0) || !std::isfinite(grid->y0))
    return FSI_ERR_INVALID_ARG;
  fsi_ctx* c = new (std::nothrow) fsi_ctx();
  if (!c) return FSI_ERR_OOM;
  c->g = *grid;
  memset(&c->x, 0, sizeof(c->x));
  if (exec) c->x = *exec;
  if ((c->x.precision != FSI_PREC_FP64 && c->x.precision != FSI_PREC_FP32 && c->x.precision != FSI_PREC_MIXED) ||
      c->x.dst_method < 0 || c->x.dst_method > 2 || (c->x.dev_alloc && !c->x.dev_free)) {
    delete c;
    return FSI_ERR_INVALID_ARG;
  }
  if (c->x.dst_method == 1 && (c->x.precision != FSI_PREC_FP32 || !gemm_dst_supported(grid->nx, grid->ny))) {
    delete c;
    return FSI_ERR_UNSUPPORTED;
  }
  if (c->x.coupling != 0 && c->x.coupling != 1) {
    delete c;
    return FSI_ERR_INVALID_ARG;
  }
  if (!(c->x.krylov_tol > 0)) c->x.krylov_tol = c->x.precision == FSI_PREC_FP64 ? 1e-10 : 1e-5;
  if (c->x.max_iters <= 0) c->x.max_iters = 50;
  if (!(c->x.tol > 0)) c->x.tol = 1e-7;
  if (c->x.history_cap <= 0) c->x.history_cap = 1 << 16;
  c->prec = c->x.precision;
  c->esz = c->prec == FSI_PREC_FP64 ? 8 : 4;
  c->fesz = c->prec == FSI_PREC_FP32 ? 4 : 8;
  c->own_stream = 0;
  if (c->x.stream) {
    c->stream = (cudaStream_t)c->x.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return FSI_ERR_CUDA;
    }
    c->own_stream = 1;
  }
  c->first_pending = 1;
  fsi_status st = create_impl(c);
  if (st == FSI_OK) st = dst_select(c);
  if (st != FSI_OK) {
    gemm_dst_free(c);
    ctx_free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return st;
  }
  *out = c;
  return FSI_OK;
}

extern "C" fsi_status fsi_add_body(fsi_ctx* c, const fsi_body_desc* b, int* body_id) {
  if (!c || !b) return FSI_ERR_INVALID_ARG;
  if (c->stage >= 1) return FSI_ERR_STATE;
  if (b->type != FSI_BODY_RIGID && b->type != FSI_BODY_TORSIONAL && b->type != FSI_BODY_DEFORMABLE &&
      b->type != FSI_BODY_DRIVEN)
    return FSI_ERR_INVALID_ARG;
  if (b->n_pts < 1 || !(b->ds > 0)) return FSI_ERR_INVALID_ARG;
  if (!c->bodies.empty() && std::fabs(b->ds - c->ds) > 1e-15 * c->ds) return FSI_ERR_UNSUPPORTED;
  BodyHost h = {};
  h.type = b->type;
  h.n = b->n_pts;
  h.off = c->nb;
  h.driver = -1;
  if (b->type == FSI_BODY_TORSIONAL) {
    if (!(b->inertia > 0) || b->stiffness < 0 || b->damping < 0) return FSI_ERR_INVALID_ARG;
    if (b->driver < 0 || b->driver > (int)c->bodies.size()) return FSI_ERR_INVALID_ARG;
    h.hx = b->hinge[0];
    h.hy = b->hinge[1];
    h.theta0 = b->theta0;
    h.inertia = b->inertia;
    h.damping = b->damping;
    h.stiffness = b->stiffness;
    h.theta = b->theta_init;
    h.phi = b->phi_init;
    h.phidot = (-b->stiffness * b->theta_init - b->damping * b->phi_init) / b->inertia;
    if (b->driver > 0) {  // hinged on a driven plate: pseudo-force moment of Eq. newtonseldg at t = 0
      const BodyHost& d = c->bodies[b->driver - 1];
      if (d.type != FSI_BODY_DRIVEN || b->theta0 != 0.0 || !(b->mass >= 0) || !std::isfinite(b->mass) ||
          !std::isfinite(b->hinge_offset) || !std::isfinite(b->cg_offset))
        return FSI_ERR_INVALID_ARG;
      h.driver = b->driver - 1;
      h.l1 = b->hinge_offset;
      h.mass = b->mass;
      h.l2 = b->cg_offset;
      double q[6];
      flapping_state(d.kin, 0.0, q);
      const double th = b->theta_init, ml = h.mass * h.l1 * h.l2;
      const double g = -h.mass * h.l2 * std::cos(q[3] + th) * q[2] - (b->inertia + ml * std::cos(th)) * q[5] -
                       ml * std::sin(th) * q[4] * q[4];
      h.phidot += g / b->inertia;
    }
    for (int j = 0; j < b->n_pts; ++j) {
      c->rigid_pts.push_back(0.0);
      c->rigid_pts.push_back(0.0);
      c->rigid_ur.push_back(0.0);
      c->rigid_ur.push_back(0.0);
    }
  } else if (b->type == FSI_BODY_DEFORMABLE) {
    if (b->n_pts < 2 || !(b->mass_per_length > 0) || !(b->bending_stiffness > 0) || !(b->stretching_stiffness > 0) ||
        b->phi_init != 0.0 || !std::isfinite(b->theta_init) || !std::isfinite(b->theta0) ||
        !std::isfinite(b->hinge[0]) || !std::isfinite(b->hinge[1]) || !std::isfinite(b->mass_per_length) ||
        !std::isfinite(b->bending_stiffness) || !std::isfinite(b->stretching_stiffness))
      return FSI_ERR_INVALID_ARG;
    h.hx = b->hinge[0];
    h.hy = b->hinge[1];
    h.theta0 = b->theta0;
    h.mu = b->mass_per_length;
    h.ei = b->bending_stiffness;
    h.ea = b->stretching_stiffness;
    h.el_off = c->ne_tot;
    const int ne = b->n_pts - 1;
    const size_t o = c->beam_chi.size();
    c->beam_chi.resize(o + 3 * ne);
    c->beam_zeta.resize(o + 3 * ne);
    c->beam_zdot.resize(o + 3 * ne);
    c->beam_ref.resize(o + 3 * ne);
    h.theta = beam_initial_state(h, b->ds, b->theta_init, &c->beam_chi[o], &c->beam_zeta[o], &c->beam_zdot[o],
                                 &c->beam_ref[o]);
    c->n_def += 1;
    c->ne_tot += ne;
    c->nd_tot += 3 * ne;
    if (3 * ne > c->nd_max) c->nd_max = 3 * ne;
    for (int j = 0; j < b->n_pts; ++j) {
      c->rigid_pts.push_back(0.0);
      c->rigid_pts.push_back(0.0);
      c->rigid_ur.push_back(0.0);
      c->rigid_ur.push_back(0.0);
    }
  } else if (b->type == FSI_BODY_DRIVEN) {
    if (!flapping_params_ok(b->kinematics) || !std::isfinite(b->s_lo) || !std::isfinite(b->hinge[0]) ||
        !std::isfinite(b->hinge[1]))
      return FSI_ERR_INVALID_ARG;
    h.hx = b->hinge[0];
    h.hy = b->hinge[1];
    for (int k = 0; k < 5; ++k) h.kin[k] = b->kinematics[k];
    h.s_lo = b->s_lo;
    for (int j = 0; j < b->n_pts; ++j) {
      c->rigid_pts.push_back(0.0);
      c->rigid_pts.push_back(0.0);
      c->rigid_ur.push_back(0.0);
      c->rigid_ur.push_back(0.0);
    }
  } else {
    if (!b->pts) return FSI_ERR_INVALID_ARG;
    h.append = b->append_to_subdomain != 0;
    for (int j = 0; j < 2 * b->n_pts; ++j) {
      c->rigid_pts.push_back(b->pts[j]);
      c->rigid_ur.push_back(b->ur ? b->ur[j] : 0.0);
    }
  }
  c->ds = b->ds;
  c->bodies.push_back(h);
  c->nb += b->n_pts;
  if (body_id) *body_id = (int)c->bodies.size() - 1;
  return FSI_OK;
}

fsi_status snap_box(const fsi_grid_desc& g, const fsi_box& b, int* i_lo_, int* i_hi_, int* j_lo_, int* j_hi_) {
  const double h = g.h;
  if (!std::isfinite(b.x_lo) || !std::isfinite(b.x_hi) || !std::isfinite(b.y_lo) || !std::isfinite(b.y_hi))
    return FSI_ERR_INVALID_ARG;
  int i_lo = (int)std::ceil((b.x_lo - g.x0) / h - 1e-9), i_hi = (int)std::floor((b.x_hi - g.x0) / h + 1e-9);
  int j_lo = (int)std::ceil((b.y_lo - g.y0) / h - 1e-9), j_hi = (int)std::floor((b.y_hi - g.y0) / h + 1e-9);
  if (i_lo < 2) i_lo = 2;
  if (j_lo < 2) j_lo = 2;
  if (i_hi > g.nx - 2) i_hi = g.nx - 2;
  if (j_hi > g.ny - 2) j_hi = g.ny - 2;
  if (i_hi <= i_lo || j_hi <= j_lo) return FSI_ERR_INVALID_ARG;
  *i_lo_ = i_lo;
  *i_hi_ = i_hi;
  *j_lo_ = j_lo;
  *j_hi_ = j_hi;
  return FSI_OK;
}

extern "C" fsi_status fsi_set_subdomain(fsi_ctx* c, const fsi_box* boxes, int n_boxes, const double* extra,
                                        int n_extra) {
  (void)extra;
  if (!c || !boxes || n_boxes < 1) return FSI_ERR_INVALID_ARG;
  if (c->stage >= 1) return FSI_ERR_STATE;
  if (n_boxes > 16 || n_extra != 0) return FSI_ERR_UNSUPPORTED;
  int sdb[16][4];
  int n_pts = 0;
  for (int k = 0; k < n_boxes; ++k) {
    const fsi_status st = snap_box(c->g, boxes[k], &sdb[k][0], &sdb[k][1], &sdb[k][2], &sdb[k][3]);
    if (st != FSI_OK) return st;
    for (int q = 0; q < k; ++q)  // boxes of a union share no vertex
      if (sdb[k][0] <= sdb[q][1] && sdb[q][0] <= sdb[k][1] && sdb[k][2] <= sdb[q][3] && sdb[q][2] <= sdb[k][3])
        return FSI_ERR_INVALID_ARG;
    n_pts += (sdb[k][1] - sdb[k][0] + 1) * (sdb[k][3] - sdb[k][2] + 1);
  }
  c->n_sdb = n_boxes;
  memcpy(c->sdb, sdb, sizeof(int) * 4 * (size_t)n_boxes);
  int i_lo = sdb[0][0], i_hi = sdb[0][1], j_lo = sdb[0][2], j_hi = sdb[0][3];
  for (int k = 1; k < n_boxes; ++k) {  // bounding box of the union
    i_lo = std::min(i_lo, sdb[k][0]);
    i_hi = std::max(i_hi, sdb[k][1]);
    j_lo = std::min(j_lo, sdb[k][2]);
    j_hi = std::max(j_hi, sdb[k][3]);
  }
  c->i_lo = i_lo;
  c->i_hi = i_hi;
  c->j_lo = j_lo;
  c->j_hi = j_hi;
  c->ni = i_hi - i_lo + 1;
  c->nj = j_hi - j_lo + 1;
  c->n_box = c->n_sd = n_pts;
  c->have_sd = 1;
  return FSI_OK;
}

// Bounding-box map and point list of a union of boxes (fsi_ctx::d_sd_map, d_sd_vert).
static fsi_status setup_union(fsi_ctx* c) {
  if (c->n_sdb <= 1) return FSI_OK;
  std::vector<int> map((size_t)c->ni * c->nj, -1), vert(2 * (size_t)c->n_box);
  int p = 0;
  for (int k = 0; k < c->n_sdb; ++k)
    for (int j = c->sdb[k][2]; j <= c->sdb[k][3]; ++j)
      for (int i = c->sdb[k][0]; i <= c->sdb[k][1]; ++i, ++p) {
        const int ii = i - c->i_lo, jj = j - c->j_lo;
        map[(size_t)jj * c->ni + ii] = p;
        vert[2 * (size_t)p] = ii;
        vert[2 * (size_t)p + 1] = jj;
      }
  if (!(c->d_sd_map = (int*)ctx_alloc(c, map.size() * sizeof(int))) ||
      !(c->d_sd_vert = (int*)ctx_alloc(c, vert.size() * sizeof(int))))
    return FSI_ERR_OOM;
  FSI_CUDA_TRY(cudaMemcpyAsync(c->d_sd_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  FSI_CUDA_TRY(cudaMemcpyAsync(c->d_sd_vert, vert.data(), vert.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  return FSI_OK;
}

// Offline stage: the operator is built (load == NULL) or read from a file written by fsi_save_operator,
// then the bodies are set up on the device.
static fsi_status precompute_impl(fsi_ctx* c, double drop_tol, const char* load) {
  NvtxRange range(load ? "fsi_load_operator" : "fsi_precompute");
  if (!c || !(drop_tol >= 0.0) || !(drop_tol < 1.0)) return FSI_ERR_INVALID_ARG;
  if (drop_tol > 0.0 && c->x.b0_method != 0) return FSI_ERR_UNSUPPORTED;
  if (c->stage >= 1) return FSI_ERR_STATE;
  if (!c->have_sd) return FSI_ERR_STATE;
  c->n_bodies = (int)c->bodies.size();
  c->nf = 2 * c->nb;
  if (c->n_bodies > 64) return FSI_ERR_UNSUPPORTED;
  const int true_e = c->x.coupling == 1;
  // appended points (Sec. 3.1.1): the fixed points of RIGID bodies flagged append_to_subdomain
  c->n_app = 0;
  c->app_pts.clear();
  if (!true_e)
    for (const BodyHost& hb : c->bodies)
      if (hb.type == FSI_BODY_RIGID && hb.append) {
        for (int j = 0; j < 2 * hb.n; ++j) c->app_pts.push_back(c->rigid_pts[2 * (size_t)hb.off + j]);
        c->n_app += hb.n;
      }
  c->n_sd = c->n_box + c->n_app;
  if (c->n_app > 0 && (drop_tol > 0.0 || load)) return FSI_ERR_UNSUPPORTED;
  // a union of boxes: the Green's-function operator (dense or filtered) and the sub-domain coupling only
  if (c->n_sdb > 1 && (c->n_app > 0 || load || true_e || c->x.b0_method != 0)) return FSI_ERR_UNSUPPORTED;
  TRY(setup_union(c));
  if (true_e) {  // true E at the body points: no B0; torsional and rigid bodies
    if (drop_tol > 0.0 || c->n_def > 0 || c->nb > 1024 || c->prec == FSI_PREC_MIXED) return FSI_ERR_UNSUPPORTED;
    if (c->x.krylov_max_iters <= 0) c->x.krylov_max_iters = 2 * c->nf + 20;
  } else if (c->nb > 0) {
    // the FSI kernel keeps the float inverse in every CTA's shared memory when it fits (nf up to ~230), and
    // otherwise distributes a block-Jacobi inverse and K over the CTAs through global memory
    const int want = c->x.fsi_solver;
    if (want < 0 || want > 2) return FSI_ERR_INVALID_ARG;
    const bool small_ok = fsi_smem_fits(c, false);
    c->fsi_big = want == 2 || (want == 0 && !small_ok);
    if (!c->fsi_big && !small_ok) return FSI_ERR_UNSUPPORTED;
    if (c->fsi_big && !fsi_smem_fits(c, true)) return FSI_ERR_UNSUPPORTED;
  }
  const size_t n2 = 2 * (size_t)c->n_sd;
  fsi_status st = FSI_OK;
  if (load && true_e) return FSI_ERR_UNSUPPORTED;
  c->drop_tol = drop_tol;
  if (true_e) {
    c->b0_seconds = 0.0;
  } else if (load) {
    const auto t0 = std::chrono::steady_clock::now();
    st = load_operator_data(c, load);
    c->b0_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  } else if (drop_tol > 0.0) {  // sparse B0' (Eq. filtereq) in the windowed column format
    st = build_b0_window(c, drop_tol);
  } else {
    if (!(c->B0 = (double*)ctx_alloc(c, n2 * n2 * 8))) return FSI_ERR_OOM;
    if (c->n_app > 0) {
      st = setup_appended(c);
      if (st == FSI_OK) st = build_appended_b0(c);
    } else {
      st = c->x.b0_method == 1 ? build_b0_columns(c) : build_b0(c);
    }
  }
  if (st != FSI_OK) return st;
  c->have_b0 = 1;
  if (c->nb > 0) {
    std::vector<BodyDev> bd;
    std::vector<BodyState> bs;
    std::vector<int> pb;
    for (size_t i = 0; i < c->bodies.size(); ++i) {
      const BodyHost& h = c->bodies[i];
      BodyDev d = {};
      d.type = h.type;
      d.off = h.off;
      d.n = h.n;
      d.hx = h.hx;
      d.hy = h.hy;
      d.theta0 = h.theta0;
      d.inertia = h.inertia;
      d.damping = h.damping;
      d.stiffness = h.stiffness;
      d.el_off = h.el_off;
      d.mu = h.mu;
      d.ei = h.ei;
      d.ea = h.ea;
      d.ca0 = std::cos(h.theta0);
      d.sa0 = std::sin(h.theta0);
      d.driver = h.driver;
      d.s_lo = h.s_lo;
      d.l1 = h.l1;
      d.mass = h.mass;
      d.l2 = h.l2;
      bd.push_back(d);
      BodyState s = {};
      s.theta = h.theta;
      s.phi = h.phi;
      s.phidot = h.phidot;
      bs.push_back(s);
      for (int j = 0; j < h.n; ++j) pb.push_back((int)i);
    }
    c->hist_cap = c->x.history_cap;
    if (!(c->d_bodies = (BodyDev*)ctx_alloc(c, bd.size() * sizeof(BodyDev))) ||
        !(c->d_state = (BodyState*)ctx_alloc(c, bs.size() * sizeof(BodyState))) ||
        !(c->d_point_body = (int*)ctx_alloc(c, pb.size() * sizeof(int))) ||
        !(c->d_rpts = (double*)ctx_alloc(c, c->rigid_pts.size() * 8)) ||
        !(c->d_rur = (double*)ctx_alloc(c, c->rigid_ur.size() * 8)) ||
        !(c->d_pidx = (int*)ctx_alloc(c, (size_t)c->nb * 4 * sizeof(int))) ||
        !(c->d_pcij = (int*)ctx_alloc(c, (size_t)c->nb * 2 * sizeof(int))) ||
        !(c->d_pw = (double*)ctx_alloc(c, (size_t)c->nb * 4 * 8)) ||
        !(c->d_sv = (double*)ctx_alloc(c, (size_t)c->nb * 2 * 8)) ||
        !(c->d_rhs = (double*)ctx_alloc(c, (size_t)c->nf * 3 * 8)) ||
        !(c->d_K = (double*)ctx_alloc(c, (size_t)c->nf * c->nf * 8)) ||
        !(c->d_f = (double*)ctx_alloc(c, (size_t)c->nf * 8)) ||
        !(c->d_Kinv = (float*)ctx_alloc(c, (size_t)c->nf * fsi_float_ld(c->nf) * 4)) ||
        !(c->d_W = (float*)ctx_alloc(c, (size_t)c->nf * fsi_float_ld(c->nf) * 4)) ||
        !(c->d_S = (float*)ctx_alloc(c, (size_t)c->nf * fsi_float_ld(c->nf) * 4)) ||
        !(c->d_T = (float*)ctx_alloc(c, (size_t)c->nf * fsi_float_ld(c->nf) * 4)) ||
        !(c->d_phase = (unsigned long long*)ctx_alloc(c, 24 * sizeof(unsigned long long))) ||
        !(c->d_part = (double*)ctx_alloc(c, (size_t)2 * 1024 * 8)) ||
        !(c->d_hist = (double*)ctx_alloc(c, (size_t)c->hist_cap * c->n_bodies * 6 * 8)))
      return FSI_ERR_OOM;
    if (c->n_app > 0) {  // Omega_0 index of every body point, then the body point of every appended index
      std::vector<int> ai(c->nb + c->n_app, -1);
      int e = 0;
      for (const BodyHost& hb : c->bodies)
        if (hb.type == FSI_BODY_RIGID && hb.append)
          for (int j = 0; j < hb.n; ++j, ++e) {
            ai[hb.off + j] = e;
            ai[c->nb + e] = hb.off + j;
          }
      if (!(c->d_app_idx = (int*)ctx_alloc(c, ai.size() * sizeof(int)))) return FSI_ERR_OOM;
      FSI_CUDA_TRY(cudaMemcpyAsync(c->d_app_idx, ai.data(), ai.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    }
    bool driven = false;
    for (const BodyHost& h : c->bodies) driven = driven || h.type == FSI_BODY_DRIVEN;
    if (driven) {  // per-step kinematics table, filled ahead of the steps by fsi_advance
      c->kin_cap = 1024;
      if (!(c->d_kin = (double*)ctx_alloc(c, (size_t)c->kin_cap * c->n_bodies * 6 * 8))) return FSI_ERR_OOM;
    }
    FSI_CUDA_TRY(cudaMemcpyAsync(c->d_bodies, bd.data(), bd.size() * sizeof(BodyDev), cudaMemcpyHostToDevice, c->stream));
    FSI_CUDA_TRY(cudaMemcpyAsync(c->d_state, bs.data(), bs.size() * sizeof(BodyState), cudaMemcpyHostToDevice, c->stream));
    FSI_CUDA_TRY(cudaMemcpyAsync(c->d_point_body, pb.data(), pb.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    FSI_CUDA_TRY(cudaMemcpyAsync(c->d_rpts, c->rigid_pts.data(), c->rigid_pts.size() * 8, cudaMemcpyHostToDevice, c->stream));
    FSI_CUDA_TRY(cudaMemcpyAsync(c->d_rur, c->rigid_ur.data(), c->rigid_ur.size() * 8, cudaMemcpyHostToDevice, c->stream));
    if (c->n_def > 0) {
      const size_t nd = (size_t)c->nd_tot;
      if (!(c->d_bchi = (double*)ctx_alloc(c, nd * 8)) || !(c->d_bzeta = (double*)ctx_alloc(c, nd * 8)) ||
          !(c->d_bzdot = (double*)ctx_alloc(c, nd * 8)) || !(c->d_bref = (double*)ctx_alloc(c, nd * 8)) ||
          !(c->d_G = (double*)ctx_alloc(c, (size_t)c->nf * c->nf * 8)))
        return FSI_ERR_OOM;
      FSI_CUDA_TRY(cudaMemcpyAsync(c->d_bchi, c->beam_chi.data(), nd * 8, cudaMemcpyHostToDevice, c->stream));
      FSI_CUDA_TRY(cudaMemcpyAsync(c->d_bzeta, c->beam_zeta.data(), nd * 8, cudaMemcpyHostToDevice, c->stream));
      FSI_CUDA_TRY(cudaMemcpyAsync(c->d_bzdot, c->beam_zdot.data(), nd * 8, cudaMemcpyHostToDevice, c->stream));
      FSI_CUDA_TRY(cudaMemcpyAsync(c->d_bref, c->beam_ref.data(), nd * 8, cudaMemcpyHostToDevice, c->stream));
    }
    if (true_e) {
      const size_t nf = (size_t)c->nf;
      if (!(c->te_w = ctx_alloc(c, (size_t)c->lvl_elems * c->esz)) ||
          !(c->te_s = ctx_alloc(c, (size_t)c->lvl_elems * c->esz)) ||
          !(c->d_te_pt = ctx_alloc(c, (size_t)c->nb * true_e_point_bytes())) ||
          !(c->d_te_r = (double*)ctx_alloc(c, nf * 8)) || !(c->d_te_p = (double*)ctx_alloc(c, nf * 8)) ||
          !(c->d_te_q = (double*)ctx_alloc(c, nf * 8)) ||
          !(c->d_te_scal = (double*)ctx_alloc(c, 8 * 8)) || !(c->d_te_ctl = (int*)ctx_alloc(c, 16 * sizeof(int))) ||
          !(c->d_te_total = (unsigned long long*)ctx_alloc(c, sizeof(unsigned long long))))
        return FSI_ERR_OOM;
      for (int k = 0; k < 2; ++k)
        if (!c->te_stream[k]) FSI_CUDA_TRY(cudaStreamCreateWithFlags(&c->te_stream[k], cudaStreamNonBlocking));
      TRY(true_e_setup(c));
      FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
      c->stage = 1;
      return FSI_OK;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = fsi_kernel_max_ctas_per_sm(c);
    if (per_sm < 1) return FSI_ERR_UNSUPPORTED;
    // two rows of the small system per CTA (at most one CTA per SM): small systems leave SMs free for
    // the kernels of other runs on the same GPU
    c->fsi_grid = c->fsi_big ? nsm : (c->nf + 1) / 2;
    if (c->fsi_grid < 8) c->fsi_grid = 8;
    if (c->fsi_grid > nsm) c->fsi_grid = nsm;
    if (c->fsi_grid < fsi_min_grid(c->nf, c->fsi_big != 0)) return FSI_ERR_UNSUPPORTED;
    if (c->fsi_big && (!(c->d_dvec = (double*)ctx_alloc(c, (size_t)c->nf * 8)) ||
                       !(c->d_rsum = (double*)ctx_alloc(c, (size_t)c->nf * 8)) ||
                       !(c->d_resf = (float*)ctx_alloc(c, (size_t)2 * c->nf * 4))))
      return FSI_ERR_OOM;
  }
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->stage = 1;
  return FSI_OK;
}

extern "C" fsi_status fsi_precompute(fsi_ctx* c, double drop_tol) { return precompute_impl(c, drop_tol, nullptr); }

extern "C" fsi_status fsi_load_operator(fsi_ctx* c, const char* path) {
  if (!path) return FSI_ERR_INVALID_ARG;
  return precompute_impl(c, 0.0, path);
}

void prof_mark(fsi_ctx* c, int cls) {
  if (c->prof_class != cls || c->prof_used >= (int)c->prof_ev.size()) return;
  cudaEventRecord(c->prof_ev[c->prof_used++], c->stream);
}

static fsi_status enqueue_step(fsi_ctx* c, int first, int capture = 0) {
  NvtxRange range(capture ? "capture step graph" : "enqueue step");
  c->launches_per_step = 0;
  TRY(launch_predictor(c, first));
  if (c->nb > 0 && c->x.coupling == 1) {
    TRY(launch_true_e(c, capture));
  } else if (c->nb > 0) {
    TRY(launch_fsi(c));
    TRY(launch_corrector(c));
  }
  return FSI_OK;
}

static fsi_status build_graph(fsi_ctx* c) {
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return FSI_ERR_CUDA;
  }
  fsi_status st = enqueue_step(c, 0, 1);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (st != FSI_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return FSI_ERR_CUDA;
  }
  if (cudaGraphInstantiate(&c->gexec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return FSI_ERR_CUDA;
  }
  c->graph = g;
  c->graph_ok = 1;
  return FSI_OK;
}

extern "C" fsi_status fsi_advance(fsi_ctx* c, int n_steps) {
  if (!c || n_steps < 0) return FSI_ERR_INVALID_ARG;
  NvtxRange range("fsi_advance");
  if (c->nb > 0 && c->stage < 1) return FSI_ERR_STATE;
  if (c->nb > 0 && !c->have_b0) return FSI_ERR_STATE;
  for (int n = 0; n < n_steps; ++n) {
    if (c->d_kin && (n == 0 || c->steps_done % c->kin_cap == 0)) {  // kinematics of the next steps
      const long long left = n_steps - n, room = c->kin_cap - c->steps_done % c->kin_cap;
      TRY(upload_kinematics(c, c->steps_done, (int)(left < room ? left : room)));
    }
    if (c->first_pending) {
      TRY(enqueue_step(c, 1));
      c->first_pending = 0;
    } else if (c->x.use_graph) {
      if (!c->graph_ok && !c->graph_failed) {
        if (build_graph(c) != FSI_OK) c->graph_failed = 1;
      }
      if (c->graph_ok) {
        FSI_CUDA_TRY(cudaGraphLaunch(c->gexec, c->stream));
      } else {
        TRY(enqueue_step(c, 0));
      }
    } else {
      TRY(enqueue_step(c, 0));
    }
    c->steps_done++;
  }
  return FSI_OK;
}

extern "C" fsi_status fsi_profile_kernel(fsi_ctx* c, int kernel_class, int n_steps, double* avg_ms,
                                         int* launches) {
  if (!c || kernel_class < KC_XF || kernel_class > KC_RING || n_steps < 1 || n_steps > 1024 || !avg_ms ||
      !launches)
    return FSI_ERR_INVALID_ARG;
  if (c->nb > 0 && c->stage < 1) return FSI_ERR_STATE;
  const int cap = 2 * 32 * n_steps;
  c->prof_ev.assign(cap, nullptr);
  fsi_status st = FSI_OK;
  for (int k = 0; k < cap; ++k)
    if (cudaEventCreate(&c->prof_ev[k]) != cudaSuccess) st = FSI_ERR_CUDA;
  c->prof_class = kernel_class;
  c->prof_used = 0;
  for (int n = 0; st == FSI_OK && n < n_steps; ++n) {
    if (c->d_kin) st = upload_kinematics(c, c->steps_done, 1);
    if (st != FSI_OK) break;
    st = enqueue_step(c, c->first_pending);
    c->first_pending = 0;
    c->steps_done++;
  }
  c->prof_class = KC_NONE;
  double sum = 0.0;
  int pairs = 0;
  if (st == FSI_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = FSI_ERR_CUDA;
  for (int k = 0; st == FSI_OK && k + 1 < c->prof_used; k += 2) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->prof_ev[k], c->prof_ev[k + 1]) != cudaSuccess) st = FSI_ERR_CUDA;
    sum += ms;
    ++pairs;
  }
  for (cudaEvent_t e : c->prof_ev)
    if (e) cudaEventDestroy(e);
  c->prof_ev.clear();
  c->prof_used = 0;
  *launches = pairs;
  *avg_ms = pairs ? sum / pairs : 0.0;
  return st;
}

extern "C" fsi_status fsi_get_phase_times(fsi_ctx* c, double* ms, int n) {
  if (!c || !ms || n < 1) return FSI_ERR_INVALID_ARG;
  for (int k = 0; k < n; ++k) ms[k] = 0.0;
  if (!c->d_phase) return FSI_OK;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  unsigned long long ns[24];
  FSI_CUDA_TRY(cudaMemcpy(ns, c->d_phase, sizeof(ns), cudaMemcpyDeviceToHost));
  for (int k = 0; k < n && k < 24; ++k) ms[k] = (double)ns[k] * 1e-6;
  return FSI_OK;
}

extern "C" fsi_status fsi_sync(fsi_ctx* c) {
  if (!c) return FSI_ERR_INVALID_ARG;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  int st = 0;
  FSI_CUDA_TRY(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  return (fsi_status)st;
}

static fsi_status read_state(fsi_ctx* c, int body, BodyState* s) {
  if (!c || body < 0 || body >= (int)c->bodies.size() || !c->d_state) return FSI_ERR_INVALID_ARG;
  fsi_status st = fsi_sync(c);
  if (st != FSI_OK && st != FSI_ERR_NOT_CONVERGED) return st;
  FSI_CUDA_TRY(cudaMemcpy(s, c->d_state + body, sizeof(BodyState), cudaMemcpyDeviceToHost));
  return st;
}

extern "C" fsi_status fsi_get_forces(fsi_ctx* c, int body, double* fx, double* fy, double* moment) {
  BodyState s;
  fsi_status st = read_state(c, body, &s);
  if (st != FSI_OK && st != FSI_ERR_NOT_CONVERGED) return st;
  if (fx) *fx = s.fx;
  if (fy) *fy = s.fy;
  if (moment) *moment = s.moment;
  return st;
}

extern "C" fsi_status fsi_read_outputs_async(fsi_ctx* c, double* out, int cap) {
  if (!c || !out || !c->d_state) return FSI_ERR_INVALID_ARG;
  const int nbody = (int)c->bodies.size();
  if (nbody == 0 || cap < 5 * nbody) return FSI_ERR_INVALID_ARG;
  // fx, fy, moment and theta, phi are two runs of consecutive doubles in every body's state record
  const size_t pitch = sizeof(BodyState), row = 5 * sizeof(double);
  const char* st = reinterpret_cast<const char*>(c->d_state);  // device address: offsets only, no access
  FSI_CUDA_TRY(cudaMemcpy2DAsync(out, row, st + offsetof(BodyState, fx), pitch, 3 * sizeof(double), nbody,
                                 cudaMemcpyDeviceToHost, c->stream));
  FSI_CUDA_TRY(cudaMemcpy2DAsync(out + 3, row, st + offsetof(BodyState, theta), pitch, 2 * sizeof(double), nbody,
                                 cudaMemcpyDeviceToHost, c->stream));
  return FSI_OK;
}

extern "C" fsi_status fsi_get_deflection(fsi_ctx* c, int body, double* theta, double* phi) {
  BodyState s;
  fsi_status st = read_state(c, body, &s);
  if (st != FSI_OK && st != FSI_ERR_NOT_CONVERGED) return st;
  if (theta) *theta = s.theta;
  if (phi) *phi = s.phi;
  return st;
}

extern "C" fsi_status fsi_get_beam_state(fsi_ctx* c, int body, double* chi, double* zeta, double* zetadot, int cap,
                                         int* n_dof) {
  if (!c || body < 0 || body >= (int)c->bodies.size()) return FSI_ERR_INVALID_ARG;
  const BodyHost& h = c->bodies[body];
  if (h.type != FSI_BODY_DEFORMABLE) return FSI_ERR_INVALID_ARG;
  const int nd = 3 * (h.n - 1);
  const size_t o = 3 * (size_t)h.el_off;
  if (n_dof) *n_dof = nd;
  if ((chi || zeta || zetadot) && cap < nd) return FSI_ERR_INVALID_ARG;
  if (!c->d_bchi) {  // before fsi_precompute: the initial state
    for (int k = 0; k < nd; ++k) {
      if (chi) chi[k] = c->beam_chi[o + k];
      if (zeta) zeta[k] = c->beam_zeta[o + k];
      if (zetadot) zetadot[k] = c->beam_zdot[o + k];
    }
    return FSI_OK;
  }
  fsi_status st = fsi_sync(c);
  if (st != FSI_OK && st != FSI_ERR_NOT_CONVERGED) return st;
  if (chi) FSI_CUDA_TRY(cudaMemcpy(chi, c->d_bchi + o, nd * 8, cudaMemcpyDeviceToHost));
  if (zeta) FSI_CUDA_TRY(cudaMemcpy(zeta, c->d_bzeta + o, nd * 8, cudaMemcpyDeviceToHost));
  if (zetadot) FSI_CUDA_TRY(cudaMemcpy(zetadot, c->d_bzdot + o, nd * 8, cudaMemcpyDeviceToHost));
  return st;
}

extern "C" fsi_status fsi_get_history(fsi_ctx* c, int body, int field, double* out, int cap, int* n) {
  if (!c || !out || !n || field < 0 || field > 5 || body < 0 || body >= (int)c->bodies.size() || !c->d_hist)
    return FSI_ERR_INVALID_ARG;
  fsi_status st = fsi_sync(c);
  if (st != FSI_OK && st != FSI_ERR_NOT_CONVERGED) return st;
  const long long done = c->steps_done;
  long long kept = done < c->hist_cap ? done : c->hist_cap;
  if (kept > cap) kept = cap;
  std::vector<double> buf((size_t)c->hist_cap * c->n_bodies * 6);
  FSI_CUDA_TRY(cudaMemcpy(buf.data(), c->d_hist, buf.size() * 8, cudaMemcpyDeviceToHost));
  for (long long k = 0; k < kept; ++k) {
    const long long step = done - kept + k;
    const long slot = (long)(step % c->hist_cap);
    out[k] = buf[((size_t)slot * c->n_bodies + body) * 6 + field];
  }
  *n = (int)kept;
  return st;
}

template <typename T>
static void to_double(const void* src, double* dst, long rows, long cols, long ld) {
  const T* s = (const T*)src;
  for (long j = 0; j < rows; ++j)
    for (long i = 0; i < cols; ++i) dst[j * cols + i] = (double)s[j * ld + i];
}

extern "C" fsi_status fsi_get_field(fsi_ctx* c, int level, int which, double* out) {
  if (!c || !out || level < 0 || level >= c->G || which < 0 || which > 1) return FSI_ERR_INVALID_ARG;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  std::vector<char> buf((size_t)c->lvl_elems * c->fesz);
  const char* base = (const char*)(which == 0 ? c->w_all : c->s_all) + (size_t)level * c->lvl_elems * c->fesz;
  FSI_CUDA_TRY(cudaMemcpy(buf.data(), base, buf.size(), cudaMemcpyDeviceToHost));
  if (c->prec == FSI_PREC_MIXED)
    to_double<f2s>(buf.data(), out, c->ny + 1, c->nx + 1, c->ps);
  else if (c->fesz == 8)
    to_double<double>(buf.data(), out, c->ny + 1, c->nx + 1, c->ps);
  else
    to_double<float>(buf.data(), out, c->ny + 1, c->nx + 1, c->ps);
  return FSI_OK;
}

extern "C" fsi_status fsi_set_field(fsi_ctx* c, int level, int which, const double* in) {
  if (!c || !in || level < 0 || level >= c->G || which < 0 || which > 1) return FSI_ERR_INVALID_ARG;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  std::vector<char> buf((size_t)c->lvl_elems * c->fesz, 0);
  for (long j = 0; j <= c->ny; ++j)
    for (long i = 0; i <= c->nx; ++i) {
      const double v = in[j * (c->nx + 1) + i];
      if (c->prec == FSI_PREC_MIXED)
        ((f2s*)buf.data())[j * c->ps + i] = f2s_from_double(v);
      else if (c->fesz == 8)
        ((double*)buf.data())[j * c->ps + i] = v;
      else
        ((float*)buf.data())[j * c->ps + i] = (float)v;
    }
  char* base = (char*)(which == 0 ? c->w_all : c->s_all) + (size_t)level * c->lvl_elems * c->fesz;
  FSI_CUDA_TRY(cudaMemcpy(base, buf.data(), buf.size(), cudaMemcpyHostToDevice));
  c->first_pending = 1;
  return FSI_OK;
}

__global__ static void k_gather_b0(const double* B0, long n2, const int64_t* rows, const int64_t* cols, int n,
                                   double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = B0[rows[k] * n2 + cols[k]];
}

extern "C" fsi_status fsi_get_operator_entries(fsi_ctx* c, const int64_t* rows, const int64_t* cols, int n,
                                               double* out) {
  if (!c || n < 0 || (n > 0 && (!rows || !cols || !out))) return FSI_ERR_INVALID_ARG;
  if (c->x.coupling == 1) return FSI_ERR_UNSUPPORTED;
  if (!c->have_b0) return FSI_ERR_STATE;
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
    if (c->Bw) st = b0_window_entries(c, dr, dc, n, dout);
    else k_gather_b0<<<(n + 255) / 256, 256, 0, c->stream>>>(c->B0, n2, dr, dc, n, dout);
    if (st != FSI_OK || cudaMemcpyAsync(out, dout, n * 8, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      st = FSI_ERR_CUDA;
  }
  ctx_dev_free(c, dr);
  ctx_dev_free(c, dc);
  ctx_dev_free(c, dout);
  return st;
}

extern "C" fsi_status fsi_get_interp(fsi_ctx* c, int64_t* idx, double* w, int cap_points) {
  if (c && c->x.coupling == 1) return FSI_ERR_UNSUPPORTED;
  if (!c || !idx || !w || cap_points < c->nb || !c->d_pidx) return FSI_ERR_INVALID_ARG;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  std::vector<int> pi((size_t)c->nb * 4);
  FSI_CUDA_TRY(cudaMemcpy(pi.data(), c->d_pidx, pi.size() * sizeof(int), cudaMemcpyDeviceToHost));
  FSI_CUDA_TRY(cudaMemcpy(w, c->d_pw, pi.size() * 8, cudaMemcpyDeviceToHost));
  for (size_t k = 0; k < pi.size(); ++k) idx[k] = pi[k];
  return FSI_OK;
}

extern "C" fsi_status fsi_get_stats(fsi_ctx* c, fsi_stats* out) {
  if (!c || !out) return FSI_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->steps_done = c->steps_done;
  out->n_sd = c->n_sd;
  out->nf = c->nf;
  out->b0_seconds = c->b0_seconds;
  out->device_bytes = c->dev_bytes;
  out->launches_per_step = c->launches_per_step;
  out->b0_nnz = c->Bw ? c->b0_nnz : (int64_t)(2 * (int64_t)c->n_sd) * (2 * (int64_t)c->n_sd);
  out->b0_window = c->Bw ? c->bw : 0;
  for (int p = 0; p < 3; ++p) {
    out->dst_gemm[p] = c->dst_gemm[p];
    out->dst_us[0][p] = c->dst_us[0][p];
    out->dst_us[1][p] = c->dst_us[1][p];
  }
  if (c->d_ctrl) {
    FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
    int ctrl[16];
    FSI_CUDA_TRY(cudaMemcpy(ctrl, c->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost));
    out->last_refreshes = ctrl[12];
    out->last_iters = ctrl[1];
    out->last_solves = ctrl[5];
    out->inverse_rebuilds = ctrl[6];
  }
  if (c->d_te_ctl) {  // true-E loops: prep + post per FSI iteration; source, 3 passes, interpolation, update
                      // per Krylov iteration
    int tctl[16];
    unsigned long long total = 0;
    FSI_CUDA_TRY(cudaMemcpy(tctl, c->d_te_ctl, sizeof(tctl), cudaMemcpyDeviceToHost));
    FSI_CUDA_TRY(cudaMemcpy(&total, c->d_te_total, sizeof(total), cudaMemcpyDeviceToHost));
    out->last_krylov_iters = tctl[5];
    out->krylov_iters_total = (int64_t)total;
    out->launches_per_step = c->launches_per_step + 2 * out->last_iters + 6 * tctl[5];
  }
  return FSI_OK;
}

// The captured step holds the kernels' arguments: drop it so that the next step captures anew.
static void drop_graph(fsi_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
  c->graph_ok = 0;
  c->graph_failed = 0;
}

extern "C" fsi_status fsi_set_phase_timing(fsi_ctx* c, int on) {
  if (!c) return FSI_ERR_INVALID_ARG;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (on && c->d_phase) FSI_CUDA_TRY(cudaMemset(c->d_phase, 0, 24 * sizeof(unsigned long long)));
  if ((on != 0) != (c->phase_on != 0)) drop_graph(c);
  c->phase_on = on != 0;
  return FSI_OK;
}

extern "C" fsi_status fsi_debug_set_wait_limit(fsi_ctx* c, unsigned spin_limit, int missing_arrivals) {
  if (!c || missing_arrivals < 0 || missing_arrivals > 1024) return FSI_ERR_INVALID_ARG;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->wait_spins = spin_limit;
  c->wait_missing = missing_arrivals;
  drop_graph(c);
  return FSI_OK;
}

extern "C" fsi_status fsi_get_small_system(fsi_ctx* c, double* out, int64_t cap, int* nf_out) {
  if (!c || !out || !nf_out) return FSI_ERR_INVALID_ARG;
  if (c->x.coupling == 1 || !c->d_K || c->steps_done == 0) return FSI_ERR_STATE;
  *nf_out = c->nf;
  const int64_t n = (int64_t)c->nf * c->nf;
  if (cap < n) return FSI_ERR_INVALID_ARG;
  FSI_CUDA_TRY(cudaStreamSynchronize(c->stream));
  FSI_CUDA_TRY(cudaMemcpy(out, c->d_K, (size_t)n * 8, cudaMemcpyDeviceToHost));
  return FSI_OK;
}

extern "C" void fsi_destroy(fsi_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  gemm_dst_free(c);
  for (int k = 0; k < 2; ++k)
    if (c->te_stream[k]) cudaStreamDestroy(c->te_stream[k]);
  ctx_free_all(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}
