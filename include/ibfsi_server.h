/*
 * ibfsi_server.h -- serving runtime of the GB300 sub-domain IB-FSI library: continuous batching of
 * independent runs on one GPU.  The paper notes that the precomputed B' serves whole parametric studies
 * (Sec. 3.4, reuse when discretisation, Re and sub-domain are unchanged); here independent runs (different
 * grids, Re and structural parameters) are admitted as device memory allows, kept resident, and advanced
 * together, one time step of every active run per server tick, each run on its own CUDA stream.
 * Same conventions as ibfsi.h: host pointers, inputs copied, status codes, no aborts.
 */
#ifndef IBFSI_SERVER_H
#define IBFSI_SERVER_H

#include "ibfsi.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One run: grid (Sec. 2.2, Sec. 5), one torsional or deformable body (Sec. 2.1, App. A; other types return
 * UNSUPPORTED), one sub-domain box (Sec. 3.1.1), the compute precision, the number of steps and a caller tag.
 * history_out: NULL, or a host array of n_steps x 6 doubles that the server fills when the run retires with
 * its per-step history (fx, fy, moment, deflection and its rate as fsi_get_history's fields 0-4, FSI
 * iterations; oldest first; rows past the steps done are left as they were).  The caller keeps it valid
 * until the run's result has been polled. */
typedef struct {
  fsi_grid_desc grid;
  fsi_body_desc body;
  fsi_box box;
  int precision;
  int n_steps;
  uint64_t tag;
  double* history_out;
} fsi_request;

/* Result of a finished run.  status: FSI_OK or the first error of the run.  Forces and deflection of the
 * last step; per-step device times (CUDA events on the run's stream, queueing behind other runs included);
 * wait_ms = submit -> admission, total_ms = submit -> retirement (host clock). */
typedef struct {
  uint64_t id, tag;
  int status, steps;
  double fx, fy, moment, theta, phi;
  double mean_step_ms, p50_step_ms, p99_step_ms;
  double wait_ms, total_ms;
} fsi_result;

typedef struct {
  int queued, active, finished;
  int admitting;     /* admitted runs whose context and B0 are being built (counted in bytes_in_use) */
  size_t bytes_in_use;
  long long ticks, run_steps;
  double cell_steps; /* sum over run steps of levels x nx x ny */
  double busy_ms;    /* host wall time spent inside ticks */
} fsi_server_stats;

typedef struct fsi_server fsi_server;

/* hbm_budget_bytes: device bytes the server may hold for admitted runs (predicted per request from its
 * grid, sub-domain and body); max_active <= 0 means no limit on the number of resident runs. */
fsi_status fsi_server_create(size_t hbm_budget_bytes, int max_active, fsi_server** out);
/* Queue a request (copied); *id receives its id.  FSI_ERR_OOM if it can never fit the budget. */
fsi_status fsi_server_submit(fsi_server* s, const fsi_request* req, uint64_t* id);
/* One tick: admit what fits, advance every active run by one step, retire runs that are done.  Admission
 * (context creation and the B0 precompute of Algorithm 1 on the run's own stream) runs on a host worker
 * thread of the server, so resident runs keep stepping while a newcomer's operator is built; a run joins
 * the active set at the first tick after its admission completed (when no run is active, the tick waits for
 * the next admission instead of returning at once).  *n_active receives the number of resident runs,
 * active or being admitted (may be NULL). */
fsi_status fsi_server_step(fsi_server* s, int* n_active);
/* Move up to cap finished results to out; *n receives the count. */
fsi_status fsi_server_poll(fsi_server* s, fsi_result* out, int cap, int* n);
fsi_status fsi_server_get_stats(fsi_server* s, fsi_server_stats* out);
/* Retire active runs (their results are discarded), drop queued requests, free everything. */
void fsi_server_destroy(fsi_server* s);

#ifdef __cplusplus
}
#endif
#endif /* IBFSI_SERVER_H */
