// Serving runtime: continuous batching of independent FSI runs on one GPU.
//
// The paper notes that a precomputed B' is reusable across parametric studies (Sec. 3.4); a serving loop
// turns that into throughput: many runs (different grids, Re, structural parameters) are resident at once.
// Each tick of fsi_server_step
//   1. takes the runs whose admission completed into the active set, and hands queued requests, in arrival
//      order, to the admission worker while their predicted device footprint fits the HBM budget; the worker
//      (a host thread of the server) creates each context on a CUDA stream of its own and runs its B0
//      precompute there, so the resident runs keep stepping meanwhile,
//   2. enqueues one time step of every active run on its own stream (captured CUDA graph), bracketed by a
//      pair of events, so the runs' kernels overlap on the device,
//   3. waits for the tick, records each run's step time, and retires runs that reached their step count,
//      keeping their results (forces, deflection, per-step latency percentiles, optionally the whole
//      history) for fsi_server_poll.
// Runs never share device buffers, so a run gives the same bits alone and in the mix.  Graph capture is
// thread-local, so the worker's CUDA calls do not interfere with a capture on the tick's thread.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>
#include "internal.h"
#include "../../include/ibfsi_server.h"

namespace {

using clk = std::chrono::steady_clock;

struct Run {
  uint64_t id;
  fsi_request req;
  fsi_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  size_t bytes = 0;
  int done = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<float> step_ms;
  clk::time_point submitted, admitted;
  int status = FSI_OK;
};

}  // namespace

struct fsi_server {
  size_t budget = 0, in_use = 0;
  int max_active = 0;
  uint64_t next_id = 1;
  std::deque<Run*> queue;
  std::vector<Run*> active;
  std::deque<fsi_result> results;
  long long ticks = 0, steps = 0;
  double cell_steps = 0.0;
  double busy_ms = 0.0;
  // admission worker: runs handed over (to_admit), runs whose context and B0 are built (admitted_runs);
  // admitting = handed over and not yet taken back by a tick
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Run*> to_admit, admitted_runs;
  int admitting = 0;
  bool stop = false;
  std::thread worker;
};

// Device bytes a request will hold: per-level fields and transform scratch, B0 and the FSI workspace.
static size_t predict_bytes(const fsi_request* r) {
  const fsi_grid_desc& g = r->grid;
  const size_t esz = r->precision == FSI_PREC_FP64 ? 8 : 4;      // transforms and right-hand sides
  const size_t fesz = r->precision == FSI_PREC_FP32 ? 4 : 8;     // level fields
  const size_t ps = ((size_t)g.nx + 1 + 7) / 8 * 8;
  const size_t lvl = ((size_t)g.ny + 1) * ps;
  const size_t slots = (size_t)g.n_levels * (r->precision == FSI_PREC_MIXED ? 2 : 1);  // right-hand sides
  size_t b = (size_t)g.n_levels * lvl * fesz * 3 + slots * lvl * esz + lvl * esz + (2 + slots) * g.nx * g.ny * esz;
  const double h = g.h;
  long i_lo = (long)std::ceil((r->box.x_lo - g.x0) / h - 1e-9), i_hi = (long)std::floor((r->box.x_hi - g.x0) / h + 1e-9);
  long j_lo = (long)std::ceil((r->box.y_lo - g.y0) / h - 1e-9), j_hi = (long)std::floor((r->box.y_hi - g.y0) / h + 1e-9);
  i_lo = std::max(i_lo, 2L);
  j_lo = std::max(j_lo, 2L);
  i_hi = std::min(i_hi, (long)g.nx - 2);
  j_hi = std::min(j_hi, (long)g.ny - 2);
  const size_t nsd = (size_t)std::max(0L, i_hi - i_lo + 1) * (size_t)std::max(0L, j_hi - j_lo + 1);
  b += 4 * nsd * nsd * 8;                               // B0 (2 n_sd)^2 doubles
  const size_t nf = 2 * (size_t)r->body.n_pts;
  b += nf * nf * (8 + 12) + 64 * 1024;                  // K, float inverses, small buffers
  if (r->body.type == FSI_BODY_DEFORMABLE) b += nf * nf * 8 + 64 * (size_t)r->body.n_pts;  // T J_d^-1 T^T, state
  return b;
}

static void retire(fsi_server* s, Run* r) {
  fsi_result out = {};
  out.id = r->id;
  out.tag = r->req.tag;
  out.status = r->status;
  out.steps = r->done;
  if (r->ctx && r->status == FSI_OK) {
    fsi_status st = fsi_get_forces(r->ctx, 0, &out.fx, &out.fy, &out.moment);
    if (st == FSI_OK) st = fsi_get_deflection(r->ctx, 0, &out.theta, &out.phi);
    if (st == FSI_OK && r->req.history_out && r->done > 0) {  // rows [step][field] from the history ring
      std::vector<double> col(r->done);
      for (int f = 0; f < 6 && st == FSI_OK; ++f) {
        int n = 0;
        st = fsi_get_history(r->ctx, 0, f, col.data(), r->done, &n);
        for (int k = 0; k < n && st == FSI_OK; ++k) r->req.history_out[(long)k * 6 + f] = col[k];
      }
    }
    out.status = st;
  }
  std::vector<float> v = r->step_ms;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    double sum = 0.0;
    for (float x : v) sum += x;
    out.mean_step_ms = sum / v.size();
    out.p50_step_ms = v[v.size() / 2];
    out.p99_step_ms = v[std::min(v.size() - 1, (size_t)std::ceil(0.99 * v.size()) - 1)];
  }
  out.wait_ms = std::chrono::duration<double, std::milli>(r->admitted - r->submitted).count();
  out.total_ms = std::chrono::duration<double, std::milli>(clk::now() - r->submitted).count();
  s->results.push_back(out);
  if (r->ev0) cudaEventDestroy(r->ev0);
  if (r->ev1) cudaEventDestroy(r->ev1);
  if (r->ctx) fsi_destroy(r->ctx);
  if (r->stream) cudaStreamDestroy(r->stream);
  s->in_use -= r->bytes;
  delete r;
}

static fsi_status admit(fsi_server* s, Run* r) {
  r->admitted = clk::now();
  if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&r->ev0) != cudaSuccess || cudaEventCreate(&r->ev1) != cudaSuccess) {
    cudaGetLastError();
    return FSI_ERR_CUDA;
  }
  fsi_exec_desc x = {};
  x.precision = r->req.precision;
  x.stream = r->stream;
  x.use_graph = 1;
  x.history_cap = r->req.history_out ? std::max(16, r->req.n_steps) : 16;
  fsi_status st = fsi_create(&r->req.grid, &x, &r->ctx);
  int bid = 0;
  if (st == FSI_OK) st = fsi_add_body(r->ctx, &r->req.body, &bid);
  if (st == FSI_OK) st = fsi_set_subdomain(r->ctx, &r->req.box, 1, nullptr, 0);
  if (st == FSI_OK) st = fsi_precompute(r->ctx, 0.0);
  return st;
}

// The admission worker: builds every handed-over run (context, body, sub-domain, B0) on the run's stream and
// hands it back with its status.
static void admission_worker(fsi_server* s) {
  for (;;) {
    Run* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [s] { return s->stop || !s->to_admit.empty(); });
      if (s->stop && s->to_admit.empty()) return;
      r = s->to_admit.front();
      s->to_admit.pop_front();
    }
    const fsi_status st = admit(s, r);
    if (st != FSI_OK) r->status = st;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->admitted_runs.push_back(r);
    }
    s->cv_done.notify_all();
  }
}

extern "C" fsi_status fsi_server_create(size_t hbm_budget_bytes, int max_active, fsi_server** out) {
  if (!out || hbm_budget_bytes == 0) return FSI_ERR_INVALID_ARG;
  fsi_server* s = new (std::nothrow) fsi_server();
  if (!s) return FSI_ERR_OOM;
  s->budget = hbm_budget_bytes;
  s->max_active = max_active > 0 ? max_active : 1 << 20;
  try {
    s->worker = std::thread(admission_worker, s);
  } catch (...) {
    delete s;
    return FSI_ERR_OOM;
  }
  *out = s;
  return FSI_OK;
}

extern "C" fsi_status fsi_server_submit(fsi_server* s, const fsi_request* req, uint64_t* id) {
  if (!s || !req || req->n_steps < 1 || req->body.n_pts < 1) return FSI_ERR_INVALID_ARG;
  if (req->body.type == FSI_BODY_RIGID && !req->body.pts) return FSI_ERR_INVALID_ARG;
  Run* r = new (std::nothrow) Run();
  if (!r) return FSI_ERR_OOM;
  r->id = s->next_id++;
  r->req = *req;
  r->req.body.pts = nullptr;  // torsional and deformable bodies are served (no host arrays to keep)
  r->req.body.ur = nullptr;
  if (req->body.type != FSI_BODY_TORSIONAL && req->body.type != FSI_BODY_DEFORMABLE) {
    delete r;
    return FSI_ERR_UNSUPPORTED;
  }
  r->bytes = predict_bytes(req);
  if (r->bytes > s->budget) {
    delete r;
    return FSI_ERR_OOM;
  }
  r->submitted = clk::now();
  s->queue.push_back(r);
  if (id) *id = r->id;
  return FSI_OK;
}

extern "C" fsi_status fsi_server_step(fsi_server* s, int* n_active) {
  if (!s) return FSI_ERR_INVALID_ARG;
  NvtxRange range("fsi_server_step");
  // 1. hand queued requests to the admission worker in arrival order while the budget allows
  {
    std::lock_guard<std::mutex> lk(s->mu);
    while (!s->queue.empty() && (int)s->active.size() + s->admitting < s->max_active &&
           s->in_use + s->queue.front()->bytes <= s->budget) {
      Run* r = s->queue.front();
      s->queue.pop_front();
      s->in_use += r->bytes;
      s->to_admit.push_back(r);
      s->admitting += 1;
    }
  }
  s->cv_work.notify_one();
  //    and take the admitted runs into the active set (with no active run, wait for the next one)
  std::deque<Run*> ready;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->active.empty() && s->admitting > 0)
      s->cv_done.wait(lk, [s] { return !s->admitted_runs.empty(); });
    ready.swap(s->admitted_runs);
    s->admitting -= (int)ready.size();
  }
  for (Run* r : ready) {
    if (r->status != FSI_OK)
      retire(s, r);
    else
      s->active.push_back(r);
  }
  // 2. one step of every active run, each on its own stream
  auto t0 = clk::now();
  for (Run* r : s->active) {
    cudaEventRecord(r->ev0, r->stream);
    const fsi_status st = fsi_advance(r->ctx, 1);
    cudaEventRecord(r->ev1, r->stream);
    if (st != FSI_OK) r->status = st;
  }
  // 3. wait, record step times, retire finished runs
  std::vector<Run*> keep;
  for (Run* r : s->active) {
    if (cudaEventSynchronize(r->ev1) != cudaSuccess) {
      cudaGetLastError();
      r->status = FSI_ERR_CUDA;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, r->ev0, r->ev1);
    r->step_ms.push_back(ms);
    r->done += 1;
    const fsi_grid_desc& g = r->req.grid;
    s->cell_steps += (double)g.n_levels * g.nx * g.ny;
    s->steps += 1;
    if (r->status == FSI_OK) {
      int dev_status = 0;
      cudaMemcpy(&dev_status, r->ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
      if (dev_status != 0) r->status = dev_status;
    }
    if (r->done >= r->req.n_steps || r->status != FSI_OK)
      retire(s, r);
    else
      keep.push_back(r);
  }
  s->active.swap(keep);
  s->busy_ms += std::chrono::duration<double, std::milli>(clk::now() - t0).count();
  s->ticks += 1;
  if (n_active) {
    std::lock_guard<std::mutex> lk(s->mu);
    *n_active = (int)s->active.size() + s->admitting;
  }
  return FSI_OK;
}

extern "C" fsi_status fsi_server_poll(fsi_server* s, fsi_result* out, int cap, int* n) {
  if (!s || !n || (cap > 0 && !out)) return FSI_ERR_INVALID_ARG;
  int k = 0;
  while (k < cap && !s->results.empty()) {
    out[k++] = s->results.front();
    s->results.pop_front();
  }
  *n = k;
  return FSI_OK;
}

extern "C" fsi_status fsi_server_get_stats(fsi_server* s, fsi_server_stats* out) {
  if (!s || !out) return FSI_ERR_INVALID_ARG;
  out->queued = (int)s->queue.size();
  out->active = (int)s->active.size();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    out->admitting = s->admitting;
  }
  out->finished = (int)s->results.size();
  out->bytes_in_use = s->in_use;
  out->ticks = s->ticks;
  out->run_steps = s->steps;
  out->cell_steps = s->cell_steps;
  out->busy_ms = s->busy_ms;
  return FSI_OK;
}

extern "C" void fsi_server_destroy(fsi_server* s) {
  if (!s) return;
  {  // the worker finishes what it was handed, then stops
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (Run* r : s->admitted_runs) s->active.push_back(r);
  s->admitted_runs.clear();
  for (Run* r : s->active) retire(s, r);
  s->active.clear();
  while (!s->queue.empty()) {
    delete s->queue.front();
    s->queue.pop_front();
  }
  delete s;
}
