// Sine-transform passes as dense sine-matrix GEMMs on the tcgen05 tensor cores (FP32 path).
//
// The 2-D DST-I solve of Sec. 3.2.1 is  w = S_y (D_A .* (S_y R S_x)) S_x  (and s likewise with D_A D_L),
// with S the symmetric matrix S[k][j] = sin(pi (j+1)(k+1) / M).  Each pass below is one GEMM, or for the
// y pass two chained GEMMs with the spectral scaling between them, and writes exactly the intermediate
// layout of the FFT passes in dst.cuh, so the two implementations are interchangeable pass by pass:
//   G1  T1[kx][y]    = sum_x R[y][x] S_x[kx][x]                 (A = R, B = S_x;   M = y,  N = kx)
//   G2  R^[ky][kx]   = sum_y S_y[ky][y] T1[kx][y]               (A = S_y, B = T1;  M = ky, N = kx)
//       W^, S^       = spectral solve of R^ (same formulas as the FFT y pass, ring terms included)
//       T2w[y][kx]   = sum_ky S_y[y][ky] W^[ky][kx], T2s likewise (A = S_y, B = W^ or S^ from shared memory)
//   G3  f[y][x]      = sum_kx S_x[x][kx] T2f[y][kx]             (A = S_x, B = T2f; M = x,  N = y)
// Products are compensated 3xTF32: each fp32 operand is split into tf32 hi + lo and the MMA chain
// accumulates hi*hi + hi*lo + lo*hi in fp32 (about 2^-21 relative per product, the accuracy class of the
// FP32 FFT); partial sums of 32 products are added in fp32 registers (see Pipe).  The sine matrices are
// split once on the host and streamed by TMA; data operands are read by the threads, split in registers
// and written to shared memory in the swizzled operand layout.
//
// Bounded waits: every mbarrier wait gives up after 2 s of wall time; the kernel then records
// FSI_ERR_TIMEOUT, stops issuing work, waits (bounded) for its own copies and MMAs in flight, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>
#include "dst.cuh"
#include "internal.h"
#include "tc.cuh"

namespace {

constexpr int kThr = 256;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kNT = 32;   // N tile of G1 and G3
constexpr int kNS13 = 4;  // operand stages of G1 and G3

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  const uint32_t a = tc::smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// Per-CTA pipeline state in shared memory.  NS operand stages and two TMEM accumulators: the MMAs of stage
// t write accumulator t % 2 from zero and the threads add it into fp32 registers one stage later ("fold"),
// so the tensor core never accumulates more than 32 products of a sum (its fp32 accumulation error would
// otherwise grow with the transform length).  TMA loads of the constant operand run NS-1 stages ahead.
constexpr int kMaxStages = 4;
struct Pipe {
  uint64_t full[kMaxStages];  // TMA tiles of stage s landed
  uint64_t done[kMaxStages];  // MMAs of stage s completed
  uint32_t tmem;              // TMEM base address
  int abort;                  // a wait gave up
  int tma_issued;             // stages whose TMA was issued (thread 0)
  int tma_seen;               // stages whose TMA completion was observed (thread 0)
  int committed;              // stages committed (thread 0)
};

template <int NS>
__device__ __forceinline__ void pipe_init(Pipe* p) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&p->full[s], 1);
      tc::mbar_init(&p->done[s], 1);
    }
    p->abort = 0;
    p->tma_issued = p->tma_seen = p->committed = 0;
    tc::fence_mbar_init();
  }
}

// Stage loop over t = 0..T-1.  tma(t, s, bar): thread 0 loads the constant operand of stage t into
// buffers s; load(t): every thread reads its share of the data operand of stage t into registers;
// store(s, regs): split and write it into buffers s; mma(t, s, acc): thread 0 issues the MMAs of stage t
// into TMEM column acc (accumulate from zero); fold(t, acc): every thread adds accumulator acc of stage t
// into its registers (and writes results at the end of a sum).  Returns false if a wait gave up.
// Buffer reuse: at stage t the MMAs of stage t-1 (and so all earlier ones) are complete before the
// barrier, so buffers t % NS (last read at t-NS) and (t-1) % NS (refilled by the TMA of stage t+NS-1)
// are free.
template <int NS, class Tma, class Load, class Store, class Mma, class Fold>
__device__ __forceinline__ bool run_pipeline(Pipe* p, int T, uint32_t acc0, uint32_t acc1, Tma tma, Load load,
                                             Store store, Mma mma, Fold fold) {
  if (threadIdx.x == 0) {
    for (int t = 0; t < NS - 1 && t < T; ++t) tma(t, t, &p->full[t]);
    p->tma_issued = T < NS - 1 ? T : NS - 1;
  }
  auto regs = load(0);
  for (int t = 0; t < T; ++t) {
    const int s = t % NS;
    store(s, regs);
    if (t + 1 < T) regs = load(t + 1);
    tc::fence_async_smem();
    if (t >= 1) {
      if (!tc::mbar_wait(&p->done[(t - 1) % NS], (uint32_t)((t - 1) / NS) & 1u, kWaitNs)) p->abort = 1;
      tc::tc_fence_after();
      if (!p->abort) fold(t - 1, (t - 1) & 1 ? acc1 : acc0);
      tc::fence_async_smem();
      tc::tc_fence_before();
    }
    __syncthreads();
    if (p->abort) return false;
    if (threadIdx.x == 0) {
      const int tn = t + NS - 1;
      if (tn < T) {
        tma(tn, tn % NS, &p->full[tn % NS]);
        p->tma_issued = tn + 1;
      }
      if (!tc::mbar_wait(&p->full[s], (uint32_t)(t / NS) & 1u, kWaitNs)) {
        p->abort = 1;
      } else {
        p->tma_seen = t + 1;
        tc::tc_fence_after();
        mma(t, s, (t & 1) ? acc1 : acc0);
        tc::mma_commit(&p->done[s]);
        p->committed = t + 1;
      }
    }
  }
  if (T > 0) {
    if (!tc::mbar_wait(&p->done[(T - 1) % NS], (uint32_t)((T - 1) / NS) & 1u, kWaitNs)) p->abort = 1;
    tc::tc_fence_after();
    if (!p->abort) fold(T - 1, (T - 1) & 1 ? acc1 : acc0);
  }
  __syncthreads();
  return !p->abort;
}

// Error path: wait (bounded) for this CTA's copies and MMAs in flight, record the status.
template <int NS>
__device__ __forceinline__ void pipe_abort_cleanup(Pipe* p, int* status) {
  if (threadIdx.x == 0) {
    dev_set_status(status, FSI_ERR_TIMEOUT);
    for (int t = p->tma_seen; t < p->tma_issued; ++t)
      tc::mbar_wait(&p->full[t % NS], (uint32_t)(t / NS) & 1u, kWaitNs / 8);
    if (p->committed > 0) {
      const int t = p->committed - 1;
      tc::mbar_wait(&p->done[t % NS], (uint32_t)(t / NS) & 1u, kWaitNs / 4);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void issue_3xtf32(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                             uint32_t idesc) {
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const uint64_t ah = tc::desc_sw128(a_hi + 32 * kk), al = tc::desc_sw128(a_lo + 32 * kk);
    const uint64_t bh = tc::desc_sw128(b_hi + 32 * kk), bl = tc::desc_sw128(b_lo + 32 * kk);
    tc::mma_tf32(d, al, bh, idesc, kk == 0 ? 0u : 1u);
    tc::mma_tf32(d, ah, bl, idesc, 1u);
    tc::mma_tf32(d, ah, bh, idesc, 1u);
  }
}

// Data tile of R rows x 32 fp32 columns held in registers between its global load and its shared store.
template <int R>
struct TileRegs {
  static constexpr int N = (R * 8 + kThr - 1) / kThr;  // float4 per thread
  float4 v[N];
};

template <int R>
__device__ __forceinline__ TileRegs<R> load_tile(const float* __restrict__ src, long ld, int r0, int nrow, int c0,
                                                 int ncol) {
  TileRegs<R> g;
#pragma unroll
  for (int q = 0; q < TileRegs<R>::N; ++q) {
    const int i = threadIdx.x + q * kThr;
    const int r = i >> 3, c = i & 7;
    const int row = r0 + r, col = c0 + 4 * c;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < R * 8 && row < nrow) {
      const float* p = src + (long)row * ld;
      if (col + 3 < ncol) {
        v = __ldcg(reinterpret_cast<const float4*>(p + col));
      } else {
        if (col < ncol) v.x = p[col];
        if (col + 1 < ncol) v.y = p[col + 1];
        if (col + 2 < ncol) v.z = p[col + 2];
      }
    }
    g.v[q] = v;
  }
  return g;
}

template <int R>
__device__ __forceinline__ void store_tile(const TileRegs<R>& g, uint8_t* hi, uint8_t* lo) {
#pragma unroll
  for (int q = 0; q < TileRegs<R>::N; ++q) {
    const int i = threadIdx.x + q * kThr;
    if (i >= R * 8) break;
    const int r = i >> 3, c = i & 7;
    float4 h, l;
    tc::split_tf32(g.v[q].x, h.x, l.x);
    tc::split_tf32(g.v[q].y, h.y, l.y);
    tc::split_tf32(g.v[q].z, h.z, l.z);
    tc::split_tf32(g.v[q].w, h.w, l.w);
    const uint32_t off = tc::sw128_off(r, c);
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
  }
}

struct Empty {};

struct G1Args {
  const float* rhs;
  long rhs_ld;
  float* T1;
  long ldT;
  int Nx, Ny, PX;
  int* status;
};

// G1: CTA (blockIdx.x, blockIdx.y) computes T1 rows kx in [32 by, +32) for y in [128 bx, +128).
// Accumulators: TMEM columns [0, 32) and [32, 64).
__global__ void __launch_bounds__(kThr, 1) k_g1(const __grid_constant__ CUtensorMap mSh,
                                                const __grid_constant__ CUtensorMap mSl, G1Args a) {
  constexpr uint32_t AB = 128 * 128, BB = kNT * 128, STAGE = 2 * AB + 2 * BB;
  extern __shared__ uint8_t smem_raw[];
  __shared__ Pipe pipe;
  uint8_t* sm = align1024(smem_raw);
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * kNT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, hf = warp >> 2;
  if (threadIdx.x == 0) {
    tc::tma_prefetch_desc(&mSh);
    tc::tma_prefetch_desc(&mSl);
  }
  pipe_init<kNS13>(&pipe);
  if (warp == 0) tc::tmem_alloc(&pipe.tmem, 64);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = pipe.tmem;
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  const uint32_t idesc = tc::idesc_tf32(128, kNT);
  float sum[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) sum[j] = 0.f;
  auto tma = [&](int t, int s, uint64_t* bar) {
    uint8_t* st = sm + s * STAGE;
    tc::mbar_arrive_expect_tx(bar, 2 * BB);
    tc::tma_load_2d(st + 2 * AB, &mSh, bar, t * 32, n0);
    tc::tma_load_2d(st + 2 * AB + BB, &mSl, bar, t * 32, n0);
  };
  auto load = [&](int t) { return load_tile<128>(a.rhs, a.rhs_ld, m0, a.Ny, t * 32, a.Nx); };
  auto store = [&](int s, const TileRegs<128>& g) {
    uint8_t* st = sm + s * STAGE;
    store_tile<128>(g, st, st + AB);
  };
  auto mma = [&](int, int s, uint32_t acc) {
    const uint32_t st = tc::smem_u32(sm + s * STAGE);
    issue_3xtf32(tmem + acc, st, st + AB, st + 2 * AB, st + 2 * AB + BB, idesc);
  };
  auto fold = [&](int, uint32_t acc) {
    float v[16];
    tc::tmem_ld16(tmem + lane_off + acc + hf * 16, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) sum[j] += v[j];
  };
  if (run_pipeline<kNS13>(&pipe, a.PX / 32, 0u, 32u, tma, load, store, mma, fold)) {
    const int y = m0 + 32 * q + lane;
    if (y < a.Ny) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int kx = n0 + hf * 16 + j;
        if (kx < a.Nx) a.T1[(long)kx * a.ldT + y] = sum[j];
      }
    }
  } else {
    pipe_abort_cleanup<kNS13>(&pipe, a.status);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

struct G3Args {
  const float* T2w;
  const float* T2s;
  long ldX;
  float* fw;
  float* fs;
  long f_ld;
  int mode;  // 0 store, 1 subtract
  int Nx, Ny, PX;
  int* status;
};

// G3: CTA (bx, by, field bz) computes f[y][x] for x in [128 bx, +128), y in [32 by, +32).
__global__ void __launch_bounds__(kThr, 1) k_g3(const __grid_constant__ CUtensorMap mSh,
                                                const __grid_constant__ CUtensorMap mSl, G3Args a) {
  constexpr uint32_t AB = 128 * 128, BB = kNT * 128, STAGE = 2 * AB + 2 * BB;
  extern __shared__ uint8_t smem_raw[];
  __shared__ Pipe pipe;
  uint8_t* sm = align1024(smem_raw);
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * kNT;
  const float* src = blockIdx.z ? a.T2s : a.T2w;
  float* dst = blockIdx.z ? a.fs : a.fw;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, hf = warp >> 2;
  if (threadIdx.x == 0) {
    tc::tma_prefetch_desc(&mSh);
    tc::tma_prefetch_desc(&mSl);
  }
  pipe_init<kNS13>(&pipe);
  if (warp == 0) tc::tmem_alloc(&pipe.tmem, 64);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = pipe.tmem;
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  const uint32_t idesc = tc::idesc_tf32(128, kNT);
  float sum[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) sum[j] = 0.f;
  auto tma = [&](int t, int s, uint64_t* bar) {
    uint8_t* st = sm + s * STAGE;
    tc::mbar_arrive_expect_tx(bar, 2 * AB);
    tc::tma_load_2d(st, &mSh, bar, t * 32, m0);
    tc::tma_load_2d(st + AB, &mSl, bar, t * 32, m0);
  };
  auto load = [&](int t) { return load_tile<kNT>(src, a.ldX, n0, a.Ny, t * 32, a.Nx); };
  auto store = [&](int s, const TileRegs<kNT>& g) {
    uint8_t* st = sm + s * STAGE;
    store_tile<kNT>(g, st + 2 * AB, st + 2 * AB + BB);
  };
  auto mma = [&](int, int s, uint32_t acc) {
    const uint32_t st = tc::smem_u32(sm + s * STAGE);
    issue_3xtf32(tmem + acc, st, st + AB, st + 2 * AB, st + 2 * AB + BB, idesc);
  };
  auto fold = [&](int, uint32_t acc) {
    float v[16];
    tc::tmem_ld16(tmem + lane_off + acc + hf * 16, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) sum[j] += v[j];
  };
  if (run_pipeline<kNS13>(&pipe, a.PX / 32, 0u, 32u, tma, load, store, mma, fold)) {
    const int x = m0 + 32 * q + lane;
    if (x < a.Nx) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int y = n0 + hf * 16 + j;
        if (y < a.Ny) {
          const long o = (long)(y + 1) * a.f_ld + 1 + x;
          if (a.mode == 0) dst[o] = sum[j];
          else dst[o] -= sum[j];
        }
      }
    }
  } else {
    pipe_abort_cleanup<kNS13>(&pipe, a.status);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

struct G2Args {
  const float* T1;
  long ldT;
  float* T2w;
  float* T2s;
  long ldX;
  int Nx, Ny, PY;
  dst::SpecParams<float> sp;
  int* status;
};

// Spectral solve of one entry, as in the FFT y pass (dst::k_ysolve): k, l are 1-based frequencies.
__device__ __forceinline__ void spectral(const dst::SpecParams<float>& sp, int k, int l, float rh, float& wt,
                                         float& st) {
  const float lam = (sp.lx[k] + sp.ly[l]) * sp.inv_h2;
  const float aw = sp.inv_dt + lam * sp.inv_2re;
  float bcs = 0.f;
  if (sp.ring) {
    const float* ring = sp.ring;
    const int l0 = l - 1;
    const float bw = sp.sx1[k] * ring[0 * sp.ring_ld + l0] + sp.sxN[k] * ring[1 * sp.ring_ld + l0] +
                     ring[2 * sp.ring_ld + (k - 1)] * sp.sy1[l] + ring[3 * sp.ring_ld + (k - 1)] * sp.syN[l];
    bcs = sp.sx1[k] * ring[4 * sp.ring_ld + l0] + sp.sxN[k] * ring[5 * sp.ring_ld + l0] +
          ring[6 * sp.ring_ld + (k - 1)] * sp.sy1[l] + ring[7 * sp.ring_ld + (k - 1)] * sp.syN[l];
    rh += bw * sp.ring_w;
    bcs *= sp.inv_h2;
  }
  wt = rh / aw;
  st = (wt + bcs) / lam;
  wt *= sp.norm;
  st *= sp.norm;
}

// G2: CTA bx owns x-frequencies kx in [16 bx, +16) and the whole y range (PY = 128 MT <= 512).  One stage
// sequence of 3 MT KB stages: forward R^ = S_y T1^T (the spectral solve writes W^ and S^ as split B operands
// into shared memory at the end of each M tile), then T2w = S_y W^, then T2s = S_y S^.
constexpr int kNT2 = 16;
template <int NS>
__global__ void __launch_bounds__(kThr, 1) k_g2(const __grid_constant__ CUtensorMap mSh,
                                                const __grid_constant__ CUtensorMap mSl, G2Args a) {
  constexpr int NT = kNT2;
  constexpr uint32_t AB = 128 * 128, BB = NT * 128, STAGE = 2 * AB + 2 * BB;
  extern __shared__ uint8_t smem_raw[];
  __shared__ Pipe pipe;
  uint8_t* sm = align1024(smem_raw);
  const int MT = a.PY / 128, KB = a.PY / 32, TP = MT * KB;
  uint8_t* bw_hi = sm + NS * STAGE;  // W^ as K-major tiles [KB][NT rows][128 B]
  uint8_t* bw_lo = bw_hi + (size_t)KB * BB;
  uint8_t* bs_hi = bw_lo + (size_t)KB * BB;  // S^
  uint8_t* bs_lo = bs_hi + (size_t)KB * BB;
  const int n0 = blockIdx.x * NT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, hf = warp >> 2;
  if (threadIdx.x == 0) {
    tc::tma_prefetch_desc(&mSh);
    tc::tma_prefetch_desc(&mSl);
  }
  pipe_init<NS>(&pipe);
  if (warp == 0) tc::tmem_alloc(&pipe.tmem, 32);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = pipe.tmem;
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  const uint32_t idesc = tc::idesc_tf32(128, NT);
  float sum[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) sum[j] = 0.f;
  auto tma = [&](int t, int s, uint64_t* bar) {
    const int r = t % TP, mt = r / KB, kb = r % KB;
    uint8_t* st = sm + s * STAGE;
    tc::mbar_arrive_expect_tx(bar, 2 * AB);
    tc::tma_load_2d(st, &mSh, bar, kb * 32, mt * 128);
    tc::tma_load_2d(st + AB, &mSl, bar, kb * 32, mt * 128);
  };
  auto load = [&](int t) {
    // data operand only in the forward phase (T1 rows kx, columns y); later phases read W^ / S^ from smem
    if (t < TP) return load_tile<NT>(a.T1, a.ldT, n0, a.Nx, (t % KB) * 32, a.Ny);
    return TileRegs<NT>{};
  };
  auto store = [&](int s, const TileRegs<NT>& g) {
    uint8_t* st = sm + s * STAGE;
    store_tile<NT>(g, st + 2 * AB, st + 2 * AB + BB);
  };
  auto mma = [&](int t, int s, uint32_t acc) {
    const int ph = t / TP, kb = (t % TP) % KB;
    const uint32_t st = tc::smem_u32(sm + s * STAGE);
    uint32_t bh, bl;
    if (ph == 0) {
      bh = st + 2 * AB;
      bl = st + 2 * AB + BB;
    } else {
      bh = tc::smem_u32(ph == 1 ? bw_hi : bs_hi) + kb * BB;
      bl = tc::smem_u32(ph == 1 ? bw_lo : bs_lo) + kb * BB;
    }
    issue_3xtf32(tmem + acc, st, st + AB, bh, bl, idesc);
  };
  auto fold = [&](int t, uint32_t acc) {
    const int ph = t / TP, r = t % TP, mt = r / KB, kb = r % KB;
    float v[8];
    tc::tmem_ld8(tmem + lane_off + acc + hf * 8, v);
#pragma unroll
    for (int j = 0; j < 8; ++j) sum[j] += v[j];
    if (kb != KB - 1) return;
    const int yk = mt * 128 + 32 * q + lane;  // ky in the forward phase, y in the inverse phases
    if (ph == 0) {
      const int l = yk + 1, kbk = yk >> 5, e = yk & 31;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int row = hf * 8 + j;
        const int k = n0 + row + 1;
        float wt = 0.f, st = 0.f;
        if (k <= a.Nx && l <= a.Ny) spectral(a.sp, k, l, sum[j], wt, st);
        const uint32_t off = (uint32_t)kbk * BB + tc::sw128_off(row, e >> 2) + (e & 3) * 4;
        float hi, lo;
        tc::split_tf32(wt, hi, lo);
        *reinterpret_cast<float*>(bw_hi + off) = hi;
        *reinterpret_cast<float*>(bw_lo + off) = lo;
        tc::split_tf32(st, hi, lo);
        *reinterpret_cast<float*>(bs_hi + off) = hi;
        *reinterpret_cast<float*>(bs_lo + off) = lo;
      }
    } else if (yk < a.Ny) {
      float4* o = reinterpret_cast<float4*>((ph == 1 ? a.T2w : a.T2s) + (long)yk * a.ldX + n0 + hf * 8);
      o[0] = make_float4(sum[0], sum[1], sum[2], sum[3]);
      o[1] = make_float4(sum[4], sum[5], sum[6], sum[7]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) sum[j] = 0.f;
  };
  if (!run_pipeline<NS>(&pipe, 3 * TP, 0u, 16u, tma, load, store, mma, fold)) pipe_abort_cleanup<NS>(&pipe, a.status);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// ---------------------------------------------------------------------------------------------------
// host side

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// tf32 rounding (nearest, ties to even) of a float's bit pattern
float tf32_rne(double v) {
  float f = (float)v;
  uint32_t b;
  memcpy(&b, &f, 4);
  if ((b & 0x7f800000u) != 0x7f800000u) {
    b += 0xFFFu + ((b >> 13) & 1u);
    b &= 0xFFFFE000u;
  }
  memcpy(&f, &b, 4);
  return f;
}

// P x P sine matrix S[k][j] = sin(pi (j+1)(k+1)/P) for j, k < P-1 (zero row and column P-1), split.
void sine_split(int P, std::vector<float>& hi, std::vector<float>& lo) {
  hi.assign((size_t)P * P, 0.f);
  lo.assign((size_t)P * P, 0.f);
  for (int k = 0; k < P - 1; ++k)
    for (int j = 0; j < P - 1; ++j) {
      const long m = ((long)(j + 1) * (k + 1)) % (2L * P);
      const double s = std::sin(M_PI * (double)m / (double)P);
      const float h = tf32_rne(s);
      hi[(size_t)k * P + j] = h;
      lo[(size_t)k * P + j] = tf32_rne(s - (double)h);
    }
}

bool encode(CUtensorMap* m, void* base, int P, int box_rows) {
  EncodeTiled enc = get_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)P, (cuuint64_t)P};
  const cuuint64_t strides[1] = {(cuuint64_t)P * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t g1_smem() { return kNS13 * (2 * 128 * 128 + 2 * kNT * 128) + 1024; }
size_t g3_smem() { return g1_smem(); }
int g2_stages(int PY) { return PY <= 256 ? 4 : 2; }
size_t g2_smem(int PY) {
  return g2_stages(PY) * (2 * 128 * 128 + 2 * kNT2 * 128) + 4 * (size_t)(PY / 32) * kNT2 * 128 + 1024;
}

}  // namespace

// Resources of the tensor-core passes of one context: split sine matrices and their TMA descriptors.
struct GemmDst {
  CUtensorMap sx32_hi, sx32_lo;    // S_x, boxes of 32 rows (G1 B operand)
  CUtensorMap sx128_hi, sx128_lo;  // S_x, boxes of 128 rows (G3 A operand)
  CUtensorMap sy128_hi, sy128_lo;  // S_y, boxes of 128 rows (G2 A operand)
};

bool gemm_dst_supported(int nx, int ny) {
  return nx >= 128 && ny >= 128 && nx <= 1024 && ny <= 512 && (nx & (nx - 1)) == 0 && (ny & (ny - 1)) == 0;
}

fsi_status gemm_dst_setup(fsi_ctx* c) {
  if (c->prec != FSI_PREC_FP32 || !gemm_dst_supported(c->nx, c->ny)) return FSI_ERR_UNSUPPORTED;
  if (!get_encoder()) {
    fsi_set_last_message("tensor-core DST: cuTensorMapEncodeTiled is not available");
    return FSI_ERR_UNSUPPORTED;
  }
  static std::once_flag attrs;
  std::call_once(attrs, [] {
    cudaFuncSetAttribute(k_g1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g1_smem());
    cudaFuncSetAttribute(k_g3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g3_smem());
    cudaFuncSetAttribute(k_g2<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g2_smem(256));
    cudaFuncSetAttribute(k_g2<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g2_smem(512));
  });
  GemmDst* g = new (std::nothrow) GemmDst();
  if (!g) return FSI_ERR_OOM;
  c->gd = g;
  const int PX = c->nx, PY = c->ny;
  std::vector<float> hi, lo;
  float *dxh, *dxl, *dyh, *dyl;
  sine_split(PX, hi, lo);
  if (!(dxh = (float*)ctx_alloc(c, hi.size() * 4)) || !(dxl = (float*)ctx_alloc(c, lo.size() * 4))) return FSI_ERR_OOM;
  FSI_CUDA_TRY(cudaMemcpy(dxh, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice));
  FSI_CUDA_TRY(cudaMemcpy(dxl, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice));
  if (PY == PX) {
    dyh = dxh;
    dyl = dxl;
  } else {
    sine_split(PY, hi, lo);
    if (!(dyh = (float*)ctx_alloc(c, hi.size() * 4)) || !(dyl = (float*)ctx_alloc(c, lo.size() * 4)))
      return FSI_ERR_OOM;
    FSI_CUDA_TRY(cudaMemcpy(dyh, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice));
    FSI_CUDA_TRY(cudaMemcpy(dyl, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice));
  }
  if (!encode(&g->sx32_hi, dxh, PX, kNT) || !encode(&g->sx32_lo, dxl, PX, kNT) ||
      !encode(&g->sx128_hi, dxh, PX, 128) || !encode(&g->sx128_lo, dxl, PX, 128) ||
      !encode(&g->sy128_hi, dyh, PY, 128) || !encode(&g->sy128_lo, dyl, PY, 128)) {
    fsi_set_last_message("tensor-core DST: tensor map encoding failed");
    return FSI_ERR_UNSUPPORTED;
  }
  return FSI_OK;
}

void gemm_dst_free(fsi_ctx* c) {
  delete c->gd;
  c->gd = nullptr;
}

fsi_status gemm_xf(fsi_ctx* c, const float* rhs) {
  G1Args a = {rhs, c->ps, (float*)c->T1, c->ldT, c->Nx, c->Ny, c->nx, c->d_status};
  const dim3 grid(c->ny / 128, c->nx / kNT);
  k_g1<<<grid, kThr, g1_smem(), c->stream>>>(c->gd->sx32_hi, c->gd->sx32_lo, a);
  FSI_CUDA_TRY(cudaGetLastError());
  return FSI_OK;
}

fsi_status gemm_ysolve(fsi_ctx* c, const dst::SpecParams<float>& sp) {
  G2Args a = {(const float*)c->T1, c->ldT, (float*)c->T2w, (float*)c->T2s, c->ldX, c->Nx, c->Ny, c->ny, sp,
              c->d_status};
  const dim3 grid(c->nx / kNT2);
  if (g2_stages(c->ny) == 4)
    k_g2<4><<<grid, kThr, g2_smem(c->ny), c->stream>>>(c->gd->sy128_hi, c->gd->sy128_lo, a);
  else
    k_g2<2><<<grid, kThr, g2_smem(c->ny), c->stream>>>(c->gd->sy128_hi, c->gd->sy128_lo, a);
  FSI_CUDA_TRY(cudaGetLastError());
  return FSI_OK;
}

fsi_status gemm_xi(fsi_ctx* c, float* fw, float* fs, int mode) {
  G3Args a = {(const float*)c->T2w, (const float*)c->T2s, c->ldX, fw, fs, c->ps, mode, c->Nx, c->Ny, c->nx,
              c->d_status};
  const dim3 grid(c->nx / 128, c->ny / kNT, 2);
  k_g3<<<grid, kThr, g3_smem(), c->stream>>>(c->gd->sx128_hi, c->gd->sx128_lo, a);
  FSI_CUDA_TRY(cudaGetLastError());
  return FSI_OK;
}
