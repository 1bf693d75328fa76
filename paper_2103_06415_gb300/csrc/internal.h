// Internal context layout and launcher declarations (not part of the C ABI).
#pragma once
#include <nvtx3/nvToolsExt.h>
#include <vector>
#include "common.cuh"

// NVTX range for the lifetime of a scope (host; a no-op unless a profiler injects an NVTX handler)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct LevelBufs {
  void* w;      // vertex vorticity [(ny+1) x ps]
  void* s;      // vertex streamfunction
  void* nprev;  // advection term of the previous step (interior entries used)
  void* rhs;    // right-hand side, interior rows stored at [j-1][i-1] with stride ps
};

struct BodyHost {
  int type, off, n;
  double hx, hy, theta0, inertia, damping, stiffness;
  double theta, phi, phidot;
  double mu, ei, ea;  // deformable: mass per length, bending and stretching stiffness
  int el_off;         // deformable: first element in the context-wide element numbering
  double kin[5];      // driven: A0, beta, sigma_t, sigma_r, f
  double s_lo;        // driven: position of point 0 along the plate
  int driver;         // torsional: index of the driven body carrying the hinge, -1 fixed hinge
  double l1, mass, l2;  // torsional with a driver: hinge offset on the driven plate, mass, centre of mass
  int append;           // rigid: the points are appended to Omega_0
};

// Device-side body record (double).  Deformable bodies: elements el_off .. el_off + n - 2, free degrees of
// freedom 3*el_off .. 3*(el_off + n - 1) - 1 (x, y, theta of nodes 1 .. n-1).
// Driven plates: (hx, hy) is the reference point, points at s_lo + j ds along (sin, -cos)(alpha1).  Torsional
// bodies with driver >= 0: hinge at l1 along that driven plate, pseudo-force moment with mass and l2.
struct BodyDev {
  int type, off, n, el_off;
  double hx, hy, theta0, inertia, damping, stiffness;
  double mu, ei, ea, ca0, sa0;  // deformable: material, cos / sin of the undeformed direction
  int driver;
  double s_lo, l1, mass, l2;
};

// 4 x 4 face windows of a point for the 3-point delta (E and E^T at an arbitrary point, Sec. 2.2): u faces
// (iu + d, ju + e) at (x_{iu+d}, y_{ju+e+1/2}) with weight w[d] * w[4 + e]; v faces (iv + d, jv + e) at
// (x_{iv+d+1/2}, y_{jv+e}) with weight w[8 + d] * w[12 + e].
struct FaceWindow {
  int iu, ju, iv, jv;
  double w[16];
};

// 3-point discrete delta in grid units (Sec. 2.2, reading R1) with explicit roundings (no contraction).
__device__ __forceinline__ double delta3_rn(double r) {
  r = fabs(r);
  if (r <= 0.5) return __ddiv_rn(__dadd_rn(1.0, sqrt(__dsub_rn(1.0, __dmul_rn(3.0, __dmul_rn(r, r))))), 3.0);
  if (r <= 1.5) {
    const double a = __dsub_rn(1.0, r);
    const double q = fmax(0.0, __dsub_rn(1.0, __dmul_rn(3.0, __dmul_rn(a, a))));
    return __ddiv_rn(__dsub_rn(__dsub_rn(5.0, __dmul_rn(3.0, r)), sqrt(q)), 6.0);
  }
  return 0.0;
}

// E0 C row stencil of velocity component comp at an Omega_0 vertex (Eq. ibsdinterp with the delta weights
// (1/6, 2/3, 1/6) x (1/2, 1/2) on the faces next to the vertex), term t < 6: u -> s at (dx in -1..1, dy =
// +-1) with weight w3[dx] dy / 2h; v -> (dx = +-1, dy in -1..1) with weight -w3[dy] dx / 2h.
__host__ __device__ __forceinline__ void e0c_stencil(int comp, int t, double inv2h, int* dx, int* dy, double* w) {
  const double w3[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
  const int d = t / 2 - 1, e = (t & 1) ? 1 : -1;
  if (comp == 0) {
    *dx = d;
    *dy = e;
    *w = w3[d + 1] * e * inv2h;
  } else {
    *dx = e;
    *dy = d;
    *w = -w3[d + 1] * e * inv2h;
  }
}

// Per-body data of one step derived from the kinematics table (FSI kernels with driven bodies): for a
// driven plate the reference point, its velocity and the plate direction; for a torsional body the hinge,
// its velocity, alpha1', the rest direction theta0 (alpha1 - pi/2 on a driver) and the coefficients of the
// pseudo-force moment g(theta) = gx cos(alpha1 + theta) + gi + gc cos(theta) + gs sin(theta).
// KB_G holds g at the current FSI iterate.
enum { KB_X = 0, KB_Y, KB_VX, KB_VY, KB_SA, KB_CA, KB_AD, KB_T0, KB_GX, KB_GI, KB_GC, KB_GS, KB_G, KB_N };

// Mutable per-body state on the device.
struct BodyState {
  double theta, phi, phidot;
  double theta_k, phi_k, r_phi, r_theta, jac;
  double fx, fy, moment;
  double theta_p;  // true-E coupling: angle of the iterate whose S produced the current f
  double kc;       // true-E coupling: (2 ds/dt) / J of the step
  double gk;       // true-E coupling: pseudo-force moment at the current iterate (hinged plates)
  double t0;       // true-E coupling: rest direction of the step (alpha1 - pi/2 on a driven plate)
};

struct fsi_ctx {
  fsi_grid_desc g;
  fsi_exec_desc x;
  int prec;  // FSI_PREC_*
  size_t esz;   // bytes per element of the transform buffers, right-hand sides and spectral tables
  size_t fesz;  // bytes per element of the level fields w, s (float, double, or a float pair in the mixed mode)
  cudaStream_t stream;
  int G, nx, ny, Nx, Ny, Mx, My;
  int logPx, logPy, r3x, r3y;  // transform lengths 2 nx = r3x 2^logPx, 2 ny = r3y 2^logPy (r3 = 1 or 3)
  long ps;        // vertex row stride (elements)
  long lvl_elems; // (ny+1)*ps
  long ldT;       // row stride of the x->y transposed buffer (>= Ny)
  long ldX;       // row stride of the y->x buffers (>= Nx)
  // fluid buffers (precision prec)
  void *w_all, *s_all, *nprev_all, *rhs_all;
  void *T1, *T2w, *T2s, *src, *ring;  // ring: 8 x ring_ld spectra
  long ring_ld;
  // tables (double)
  double *lx, *ly, *sx1, *sxN, *sy1, *syN;
  void *lxT, *lyT, *sx1T, *sxNT, *sy1T, *syNT;  // the same tables in the context precision
  void *twx, *twy;  // complex twiddles in precision prec (length Lx, Ly)
  // sub-domain: one vertex box, or a union of n_sdb disjoint boxes (reading R16), whose points are numbered
  // box by box; i_lo .. j_hi, ni, nj then describe the bounding box of the union, d_sd_map holds the Omega_0
  // index of every bounding-box vertex (-1: not in Omega_0) and d_sd_vert the bounding-box vertex (i, j) of
  // every Omega_0 point (both NULL for one box, whose numbering is row by row over the box)
  int have_sd;
  int i_lo, i_hi, j_lo, j_hi, ni, nj, n_sd;
  int n_sdb;
  int sdb[16][4];  // i_lo, i_hi, j_lo, j_hi of every box (grid vertex indices)
  int* d_sd_map;
  int* d_sd_vert;
  // appended points (exact points of RIGID bodies flagged append, Sec. 3.1.1): unknowns n_box .. n_sd - 1 of
  // each component follow the box's n_box = ni * nj points; their face windows, the Omega_0 index of every
  // body point (-1: interpolated by P), and the vertex box their corrector source covers
  int n_box, n_app;
  std::vector<double> app_pts;
  FaceWindow* d_app_win;
  int* d_app_idx;
  int app_box[4];
  double* B0;  // (2 n_sd)^2 row-major, double (NULL when the sparse B0' is used)
  double* Bw;  // sparse B0' in the windowed column format of b0_sparse.cu, or NULL
  int bw;      // window half-width of Bw (Omega_0 points)
  long long b0_nnz;  // kept entries of B0' (sparse build)
  double drop_tol;    // filter of the operator in use (0: dense)
  double* d_factor;  // (2 n_sd)^2 lower Cholesky factor of B0 + tau I (fsi_factor_operator), or NULL
  int have_b0;
  double b0_seconds;
  // bodies
  std::vector<BodyHost> bodies;
  std::vector<double> rigid_pts, rigid_ur;  // [nb*2] (zeros for torsional points)
  int nb, nf, n_bodies;
  double ds;
  BodyDev* d_bodies;
  BodyState* d_state;
  int* d_point_body;  // body index per point
  double *d_rpts, *d_rur;
  // FSI workspace
  int* d_pidx;     // [nb*4] Omega_0 point index
  int* d_pcij;     // [nb*2] hat cell (ci, cj) of every point
  double* d_pw;    // [nb*4]
  double* d_sv;    // [nb*2] torsional S entries (Q_j R)
  double* d_rhs;   // [nf]
  double* d_K;     // [nf*nf]
  double* d_f;     // [nf]
  float* d_Kinv;   // [nf][ldx] float inverse of K used for iterative refinement (ldx: fsi_float_ld)
  float* d_W;      // [nf][ldx] second float-inverse buffer (Newton-Schulz ping-pong)
  float* d_S;      // [nf][ldx] float copy of K
  float* d_T;      // [nf][ldx] scratch: X K, or the inverse Cholesky factor
  double* d_part;  // [2*fsi_grid] per-CTA maxima
  int* d_ctrl;     // FSI control words (see fsi.cu)
  unsigned long long* d_phase;  // [8] accumulated FSI kernel phase times (ns)
  int* d_status;
  // deformable bodies (device state, FP64): chi, zeta, zetadot per free dof; per element the chord
  // rotation and direction at chi_n (reference for the rotation increment); G = columns of T J_d^-1 T^T
  // for the small system ([nf][nf], column-major, zero outside deformable blocks)
  int n_def, nd_tot, ne_tot, nd_max;
  std::vector<double> beam_chi, beam_zeta, beam_zdot, beam_ref;
  double *d_bchi, *d_bzeta, *d_bzdot, *d_bref, *d_G;
  // true-E coupling (true_e.cu): level-0 w, s of the operator application (zero ring), point face windows,
  // CG vectors r, p and q = K p, scalars, control words, CG iterations since creation, capture streams of the loops
  void *te_w, *te_s;
  void* d_te_pt;
  double *d_te_r, *d_te_p, *d_te_q, *d_te_scal;
  int* d_te_ctl;
  unsigned long long* d_te_total;
  cudaStream_t te_stream[2];
  // prescribed kinematics: [kin_cap][n_bodies][6] per step (X1, X1', X1'', alpha1, alpha1', alpha1'' at the
  // step's end time, driven bodies only; slot = step mod kin_cap), NULL without driven bodies
  double* d_kin;
  int kin_cap;
  double* d_hist;  // [cap][n_bodies][6]
  int hist_cap;
  long long steps_done;
  int max_iters_seen;
  int fsi_grid;  // CTAs of the cooperative FSI kernel
  int fsi_big;   // 1: the distributed variant of the FSI kernel (block-Jacobi inverse and K in global memory)
  double* d_dvec;  // distributed variant: [nf] corrections d = X r shared between the CTAs
  double* d_rsum;  // distributed variant: [nf] absolute row sums of K (rebuild of the inverse)
  float* d_resf;   // distributed variant: [2][nf] float copies of the residual rows (by solve parity)
  // bounded cross-CTA wait of the FSI kernel (fsi_debug_set_wait_limit): poll limit (0: default) and
  // arrivals it waits for that never come (0 in normal runs)
  unsigned wait_spins;
  int wait_missing;
  // graph
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  int graph_ok, graph_failed;
  int own_stream;     // stream created by the library (caller passed NULL)
  int phase_on;  // in-kernel phase timers of the FSI kernel (fsi_set_phase_timing), off by default
  int first_pending;  // next step uses N^{n-1} := N^n (first step, or fields were overwritten)
  int stage;          // 0 = setup, 1 = precomputed
  // live kernel timing: events around every launch of one kernel class (eager steps only)
  int prof_class;
  std::vector<cudaEvent_t> prof_ev;
  int prof_used;
  int launches_per_step;
  // sine-transform passes: dst_gemm[p] = 1 runs pass p (0 forward x, 1 y solve, 2 inverse x) as a
  // tensor-core GEMM (dst_gemm.cu) instead of the FFT pass; dst_us = autotuner timings [FFT, GEMM][pass]
  int dst_gemm[3];
  double dst_us[2][3];
  struct GemmDst* gd;
  size_t dev_bytes;
  std::vector<void*> allocs;  // buffers held for the context's lifetime (through ctx_dev_malloc)
};

// One Omega_0 box of a B0 build.  Several boxes on one grid are built together; their matrices are stored
// one after another, box k's (2 n_sd)^2 row-major block starting at out_off.
struct B0Box {
  int i_lo, j_lo, ni, nj, n_sd, pad;
  long row_off;  // first unknown of this box in the concatenated unknown list (prefix sum of 2 n_sd)
  long out_off;  // first entry of this box's matrix (prefix sum of (2 n_sd)^2)
  long tab_off;  // first entry of this box's stencil tables (Green's-function method)
};

// B0[(ca, ja, ia)][(cb, jb, ib)] of points at box vertices (ia, ja), (ib, jb) from the 16 stencil tables of
// that box (b0.cu k_tables; nx2 = 2 ni - 1, per = nx2 (2 nj - 1) entries per table), in the rounding order of
// the dense fill: (T-- - T-+) - (T+- - T++).
__device__ __forceinline__ double b0_entry(const double* __restrict__ tab, long per, int nx2, int ni, int nj,
                                           int ca, int ja, int ia, int cb, int jb, int ib) {
  const double* t = tab + (long)((ca * 2 + cb) * 4) * per;
  const long r1 = (long)(ja - jb + nj - 1) * nx2, r2 = (long)(ja + jb) * nx2;
  const int D = ia - ib + ni - 1, S = ia + ib;
  const double U = t[r1 + D] - t[2 * per + r2 + D];
  const double V = t[per + r1 + S] - t[3 * per + r2 + S];
  return U - V;
}

// Box vertex (i, j) of Omega_0 point p: row by row over one box of ni columns, or from the point list of a
// union (vert: (i, j) of every point in its bounding box; NULL for one box).
__host__ __device__ __forceinline__ void sd_vertex(const int* vert, int ni, int p, int* i, int* j) {
  if (vert) {
    *i = vert[2 * p];
    *j = vert[2 * p + 1];
  } else {
    *j = p / ni;
    *i = p - *j * ni;
  }
}

// Entry (row, col) of the sparse B0' in the windowed column format of b0_sparse.cu (unknown ordering of
// B0: the n_sd x-components, then the n_sd y-components; points as sd_vertex numbers them): column col
// keeps, for each component of the row, the (2w+1)^2 box vertices within w of its own point (zero where a
// vertex is not in Omega_0).
__host__ __device__ __forceinline__ double b0w_lookup(const double* Wv, int w, int ni, int n_sd, long row, long col,
                                                      const int* vert = nullptr) {
  const int ca = row >= n_sd, cb = col >= n_sd;
  const int pa = (int)(row - (long)ca * n_sd), pb = (int)(col - (long)cb * n_sd);
  int ia, ja, ib, jb;
  sd_vertex(vert, ni, pa, &ia, &ja);
  sd_vertex(vert, ni, pb, &ib, &jb);
  const int dj = ja - jb, di = ia - ib;
  if (dj > w || dj < -w || di > w || di < -w) return 0.0;
  const long side = 2 * w + 1;
  return Wv[col * 2 * side * side + ca * side * side + (dj + w) * side + (di + w)];
}

// box holding the global unknown u (boxes sorted by row_off)
__device__ __forceinline__ int b0_find_box(const B0Box* bx, int n, long u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bx[mid].row_off <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Fills row_off and out_off from the box order; returns the total number of matrix entries.
inline long b0_layout(std::vector<B0Box>& boxes) {
  long rows = 0, entries = 0;
  for (B0Box& b : boxes) {
    b.n_sd = b.ni * b.nj;
    b.row_off = rows;
    b.out_off = entries;
    rows += 2L * b.n_sd;
    entries += 4L * b.n_sd * b.n_sd;
  }
  return entries;
}

// the context's own Omega_0 box (without appended points)
inline B0Box ctx_box(const fsi_ctx* c) {
  B0Box b = {};
  b.i_lo = c->i_lo;
  b.j_lo = c->j_lo;
  b.ni = c->ni;
  b.nj = c->nj;
  b.n_sd = c->ni * c->nj;
  return b;
}

// Snap a box to grid vertices and clip it to >= 2 cells from the boundary; FSI_ERR_INVALID_ARG if empty.
fsi_status snap_box(const fsi_grid_desc& g, const fsi_box& b, int* i_lo, int* i_hi, int* j_lo, int* j_hi);

// fluid.cu
fsi_status launch_predictor(fsi_ctx* c, int first);
fsi_status launch_corrector(fsi_ctx* c);
fsi_status launch_level_solve(fsi_ctx* c, int g, const void* rhs, void* w, void* s, int use_ring, int mode);
// fsi.cu
fsi_status launch_fsi(fsi_ctx* c);
// kinematics.cu
bool flapping_params_ok(const double* k);
void flapping_state(const double* k, double t, double* out);
fsi_status upload_kinematics(fsi_ctx* c, long long first, int n);
// true_e.cu
fsi_status launch_true_e(fsi_ctx* c, int capture);
fsi_status true_e_setup(fsi_ctx* c);
size_t true_e_point_bytes();
// b0.cu
fsi_status build_b0(fsi_ctx* c);
fsi_status b0_green(fsi_ctx* c, std::vector<B0Box>& boxes, double* out);
fsi_status b0_green_tables(fsi_ctx* c, std::vector<B0Box>& boxes, double** tab_out);
// b0_sparse.cu
fsi_status build_b0_window(fsi_ctx* c, double drop_tol);
fsi_status b0_window_entries(fsi_ctx* c, const int64_t* d_rows, const int64_t* d_cols, int n, double* d_out);
// appended.cu
fsi_status setup_appended(fsi_ctx* c);       // face windows and indices of the appended points
fsi_status build_appended_b0(fsi_ctx* c);    // B0 with appended points (box part by the chosen method)
fsi_status launch_appended_source(fsi_ctx* c);  // corrector source of the appended points' stress
// operator_io.cu
fsi_status load_operator_data(fsi_ctx* c, const char* path);
// b0_columns.cu
fsi_status build_b0_columns(fsi_ctx* c);
fsi_status b0_columns(fsi_ctx* c, std::vector<B0Box>& boxes, double* out);

// dst_gemm.cu
bool gemm_dst_supported(int nx, int ny);
fsi_status gemm_dst_setup(fsi_ctx* c);
void gemm_dst_free(fsi_ctx* c);
fsi_status gemm_xf(fsi_ctx* c, const float* rhs);
namespace dst { template <typename T> struct SpecParams; }
fsi_status gemm_ysolve(fsi_ctx* c, const dst::SpecParams<float>& sp);
fsi_status gemm_xi(fsi_ctx* c, float* fw, float* fs, int mode);

void* ctx_alloc(fsi_ctx* c, size_t bytes);
// One device buffer through the context's allocator (fsi_exec_desc.dev_alloc) or cudaMalloc; returned by
// ctx_dev_free (NULL is a no-op).  cudaErrorMemoryAllocation when the allocator gives nothing or a pointer
// that is not 256-byte aligned.
cudaError_t ctx_dev_malloc(const fsi_ctx* c, void** p, size_t bytes);
void ctx_dev_free(const fsi_ctx* c, void* p);

// kernel classes for fsi_profile_kernel
enum { KC_NONE = 0, KC_XF = 1, KC_YSOLVE = 2, KC_XI = 3, KC_FSI = 4, KC_RHS = 5, KC_SRC = 6, KC_RING = 7 };
void prof_mark(fsi_ctx* c, int cls);  // records one event if cls is being profiled
