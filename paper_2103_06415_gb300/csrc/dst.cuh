// Batched DST-I passes built on a shared-memory Stockham FFT (radix 4, one radix-2 stage when the log2 of the
// power-of-two part is odd, one radix-3 stage for lengths 3 * 2^k).  The DST-I of two real rows x1, x2 of length N = M-1 is read off one complex FFT of length
// L = 2M of the packed odd extension z = (x1 + i x2) extended oddly about 0 and M:
//   X1_k = -Im(Z_k)/2,  X2_k = Re(Z_k)/2,  k = 1..N,
// with X_k = sum_j x_j sin(pi j k / M) (unnormalised; the inverse is (2/M) times the same transform).
// The 2-D DST diagonalises C^T C and A (Sec. 3.2.1), so a Poisson-type solve is
//   forward x (pass XF) -> forward y, diagonal scaling, inverse y (pass Y) -> inverse x (pass XI),
// with the x <-> y transposition folded into the stores of passes XF and Y.
#pragma once
#include "common.cuh"

namespace dst {

// Transform lengths L = R3 * 2^logP with R3 = 1 or 3 (DST-I lengths N = L/2 - 1 for grids of 2^k or 3 * 2^k
// cells).  The power-of-two part is done by radix-4 stages (one radix-2 stage when logP is odd); with R3 = 3 a
// final radix-3 stage follows (ns = 2^logP, inputs and outputs at the same three positions j, j + P, j + 2P).
//
// Twiddle table of length L in stage order: entry p holds exp(-2 pi i m / L) with m = twiddle_exponent(p,
// logP, R3).  A radix-4 stage with ns = 4^s > 1 (s >= 1) reads its three twiddles w_r(k) = exp(-2 pi i r k /
// (4 ns)), r = 1..3, k < ns, from the block at ns - 4, laid out [r - 1][k]; a radix-2 stage (odd logP) reads
// exp(-2 pi i k / P), k < P/2, from the block at P/2 - 4; the radix-3 stage reads exp(-2 pi i r k / L),
// r = 1, 2, k < P, from the block at P - 4, laid out [r - 1][k].  The threads of a warp read consecutive k (or
// the same k), so these shared-memory loads are free of bank conflicts, which the natural-order table (index
// r k L/(4 ns), a power-of-two stride) is not.  The blocks fill L - 4 entries.
__host__ __device__ inline int twiddle_exponent(int p, int logP, int R3 = 1) {
  for (int logNs = 2; logP - logNs >= 2; logNs += 2) {
    const int ns = 1 << logNs;
    const int q = p - (ns - 4);
    if (q < 3 * ns) return (q / ns + 1) * (((q % ns) * R3) << (logP - logNs - 2));
  }
  const int P = 1 << logP;
  if (logP & 1) {
    const int q = p - ((P >> 1) - 4);
    if (q >= 0 && q < (P >> 1)) return q * R3;
  }
  if (R3 == 3) {
    const int q = p - (P - 4);
    if (q >= 0 && q < 2 * P) return (q / P + 1) * (q % P);
  }
  return 0;
}

// Split a transform length L into R3 * 2^logP (R3 = 1 or 3, logP >= 4); false for other lengths.
__host__ __device__ inline bool split_length(int L, int* logP, int* R3) {
  int r = 1;
  if (L % 3 == 0) {
    r = 3;
    L /= 3;
  }
  if (L < 16 || (L & (L - 1)) != 0) return false;
  int k = 0;
  while ((1 << k) < L) ++k;
  *logP = k;
  *R3 = r;
  return true;
}

// Butterfly b of a stage splits into the transform f it belongs to and its index j inside the transform,
// with Lr = R3 * 2^logLr butterflies per transform.
template <int R3>
__host__ __device__ __forceinline__ void stage_index(int b, int logLr, int* f, int* j) {
  const int q = b >> logLr;
  const int fv = R3 == 1 ? q : q / 3;
  *f = fv;
  *j = b - ((fv * R3) << logLr);
}

// The butterflies of one stage, split into a load (from the stage's input, which a barrier separates from
// the stores) and a compute-and-store, so that a host program can run the same code over all butterflies to
// check indices and results.  buf holds the transforms back to back (transform f at f * L).
template <typename T, int R3>
__host__ __device__ __forceinline__ void r4_load(const typename C2<T>::t* buf, int L, int logP, int b,
                                                 typename C2<T>::t* a) {
  const int logLr = logP - 2, Lr = R3 << logLr;
  int f, j;
  stage_index<R3>(b, logLr, &f, &j);
  const typename C2<T>::t* x = buf + (long)f * L;
#pragma unroll
  for (int r = 0; r < 4; ++r) a[r] = x[j + r * Lr];
}

template <typename T, int R3>
__host__ __device__ __forceinline__ void r4_store(typename C2<T>::t* buf, int L, int logP, int logNs, int b,
                                                  const typename C2<T>::t* tw, typename C2<T>::t* a) {
  using c2 = typename C2<T>::t;
  const int logLr = logP - 2;
  int f, j;
  stage_index<R3>(b, logLr, &f, &j);
  const int k = j & ((1 << logNs) - 1);
  if (logNs > 0) {
    const c2* tws = tw + ((1 << logNs) - 4) + k;  // stage block [r - 1][k]
#pragma unroll
    for (int r = 1; r < 4; ++r) {
      const c2 w = tws[(r - 1) << logNs];
      const T re = a[r].x * w.x - a[r].y * w.y;
      const T im = a[r].x * w.y + a[r].y * w.x;
      a[r].x = re;
      a[r].y = im;
    }
  }
  const T a0x = a[0].x + a[2].x, a0y = a[0].y + a[2].y;
  const T a1x = a[0].x - a[2].x, a1y = a[0].y - a[2].y;
  const T a2x = a[1].x + a[3].x, a2y = a[1].y + a[3].y;
  const T dx = a[1].x - a[3].x, dy = a[1].y - a[3].y;  // (d)(-i) = (dy, -dx)
  c2* x = buf + (long)f * L;
  const int o = ((j >> logNs) << (logNs + 2)) + k;
  const int ns = 1 << logNs;
  if (sizeof(T) == 4 && logNs == 0) {  // the four outputs are adjacent: two 16-byte stores
    float4* x4 = reinterpret_cast<float4*>(x + o);
    x4[0] = make_float4(a0x + a2x, a0y + a2y, a1x + dy, a1y - dx);
    x4[1] = make_float4(a0x - a2x, a0y - a2y, a1x - dy, a1y + dx);
    return;
  }
  x[o].x = a0x + a2x;
  x[o].y = a0y + a2y;
  x[o + ns].x = a1x + dy;
  x[o + ns].y = a1y - dx;
  x[o + 2 * ns].x = a0x - a2x;
  x[o + 2 * ns].y = a0y - a2y;
  x[o + 3 * ns].x = a1x - dy;
  x[o + 3 * ns].y = a1y + dx;
}

template <typename T, int R3>
__host__ __device__ __forceinline__ void r2_load(const typename C2<T>::t* buf, int L, int logP, int b,
                                                 typename C2<T>::t* a) {
  const int logLr = logP - 1, Lr = R3 << logLr;
  int f, j;
  stage_index<R3>(b, logLr, &f, &j);
  const typename C2<T>::t* x = buf + (long)f * L;
  a[0] = x[j];
  a[1] = x[j + Lr];
}

template <typename T, int R3>
__host__ __device__ __forceinline__ void r2_store(typename C2<T>::t* buf, int L, int logP, int logNs, int b,
                                                  const typename C2<T>::t* tw, typename C2<T>::t* a) {
  using c2 = typename C2<T>::t;
  const int logLr = logP - 1;
  int f, j;
  stage_index<R3>(b, logLr, &f, &j);
  const int k = j & ((1 << logNs) - 1);
  c2 a0 = a[0], a1 = a[1];
  if (logNs > 0) {
    const c2 w = tw[(1 << (logP - 1)) - 4 + k];  // logNs = logP - 1: the radix-2 stage of an odd logP
    const T re = a1.x * w.x - a1.y * w.y;
    const T im = a1.x * w.y + a1.y * w.x;
    a1.x = re;
    a1.y = im;
  }
  c2* x = buf + (long)f * L;
  const int o = ((j >> logNs) << (logNs + 1)) + k;
  x[o].x = a0.x + a1.x;
  x[o].y = a0.y + a1.y;
  x[o + (1 << logNs)].x = a0.x - a1.x;
  x[o + (1 << logNs)].y = a0.y - a1.y;
}

// Radix-3 stage (the last one, ns = P = 2^logP): butterfly j of transform f takes x[j], x[j + P], x[j + 2P],
// twists the second and third by w^k, w^2k (w = exp(-2 pi i / L), k = j) and writes back to the same places:
// with s = a1 + a2, d = a1 - a2, t = a0 - s/2 and c = sqrt(3)/2 the outputs are a0 + s, t - i c d, t + i c d.
template <typename T>
__host__ __device__ __forceinline__ void r3_load(const typename C2<T>::t* buf, int L, int logP, int b,
                                                 typename C2<T>::t* a) {
  const int P = 1 << logP;
  const int f = b >> logP, j = b & (P - 1);
  const typename C2<T>::t* x = buf + (long)f * L;
  a[0] = x[j];
  a[1] = x[j + P];
  a[2] = x[j + 2 * P];
}

template <typename T>
__host__ __device__ __forceinline__ void r3_store(typename C2<T>::t* buf, int L, int logP, int b,
                                                  const typename C2<T>::t* tw, typename C2<T>::t* a) {
  using c2 = typename C2<T>::t;
  const int P = 1 << logP;
  const int f = b >> logP, k = b & (P - 1);
  const c2 w1 = tw[P - 4 + k], w2 = tw[2 * P - 4 + k];
  const T b1x = a[1].x * w1.x - a[1].y * w1.y, b1y = a[1].x * w1.y + a[1].y * w1.x;
  const T b2x = a[2].x * w2.x - a[2].y * w2.y, b2y = a[2].x * w2.y + a[2].y * w2.x;
  const T sx = b1x + b2x, sy = b1y + b2y, dx = b1x - b2x, dy = b1y - b2y;
  const T tx = a[0].x - T(0.5) * sx, ty = a[0].y - T(0.5) * sy;
  const T c = T(0.86602540378443864676);  // sqrt(3) / 2
  c2* x = buf + (long)f * L;
  x[k].x = a[0].x + sx;
  x[k].y = a[0].y + sy;
  x[k + P].x = tx + c * dy;   // t - i c d
  x[k + P].y = ty - c * dx;
  x[k + 2 * P].x = tx - c * dy;  // t + i c d
  x[k + 2 * P].y = ty + c * dx;
}

// The passes below copy the table into shared memory before their first barrier, so the stages read it
// there.  A CTA transforms nf = 4 PER blockDim / 2^logP transforms of length L = R3 2^logP: PER R3 radix-4
// butterflies (2 PER R3 radix-2, 4 PER radix-3) per thread and stage.
template <typename T, int PER, int R3 = 1>
__device__ __forceinline__ void block_fft(typename C2<T>::t* buf, int L, int logP,
                                          const typename C2<T>::t* __restrict__ tw) {
  using c2 = typename C2<T>::t;
  const int nthr = blockDim.x, tid = threadIdx.x;
  int logNs = 0;
  int rem = logP;
  while (rem > 0) {
    if (rem >= 2) {
      c2 v[4 * PER * R3];
#pragma unroll
      for (int q = 0; q < PER * R3; ++q) r4_load<T, R3>(buf, L, logP, tid + q * nthr, &v[4 * q]);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < PER * R3; ++q) r4_store<T, R3>(buf, L, logP, logNs, tid + q * nthr, tw, &v[4 * q]);
      __syncthreads();
      logNs += 2;
      rem -= 2;
    } else {
      c2 v[4 * PER * R3];
#pragma unroll
      for (int q = 0; q < 2 * PER * R3; ++q) r2_load<T, R3>(buf, L, logP, tid + q * nthr, &v[2 * q]);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 2 * PER * R3; ++q) r2_store<T, R3>(buf, L, logP, logNs, tid + q * nthr, tw, &v[2 * q]);
      __syncthreads();
      logNs += 1;
      rem -= 1;
    }
  }
  if (R3 == 3) {
    c2 v[12 * PER];
#pragma unroll
    for (int q = 0; q < 4 * PER; ++q) r3_load<T>(buf, L, logP, tid + q * nthr, &v[3 * q]);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4 * PER; ++q) r3_store<T>(buf, L, logP, tid + q * nthr, tw, &v[3 * q]);
    __syncthreads();
  }
}

// Copies the twiddles to tws when the launch gave the kernel room for them (dynamic shared memory of at
// least end_bytes, tws + L being the end of that area) and returns the table the stages should read.
template <typename T>
__device__ __forceinline__ const typename C2<T>::t* stage_twiddles(typename C2<T>::t* tws,
                                                                   const typename C2<T>::t* __restrict__ tw, int L,
                                                                   size_t end_bytes) {
  unsigned dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  if ((size_t)dyn < end_bytes) return tw;
  for (int m = threadIdx.x; m < L; m += blockDim.x) tws[m] = tw[m];
  return tws;
}

// Dynamic shared memory of a pass: its buffers (base_elems complex entries) plus the twiddles when the sum
// stays within limit_bytes.
template <typename T>
inline size_t pass_smem(size_t base_elems, int L, size_t limit_bytes = 200 * 1024) {
  const size_t e = sizeof(typename C2<T>::t);
  return (base_elems + L) * e <= limit_bytes ? (base_elems + L) * e : base_elems * e;
}

// Pack rows r0 (real part) and r1 (imag part) of length N into the odd extension in buffer f.
// Rows beyond nrows read as zero.  Caller syncs afterwards.
template <typename T>
__device__ __forceinline__ void zero_ends(typename C2<T>::t* buf, int nf, int L) {
  const int M = L >> 1;
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    buf[(long)f * L].x = 0;
    buf[(long)f * L].y = 0;
    buf[(long)f * L + M].x = 0;
    buf[(long)f * L + M].y = 0;
  }
}

template <typename T>
__device__ __forceinline__ void put_pair(typename C2<T>::t* z, int L, int n, T a, T b) {
  z[n + 1].x = a;
  z[n + 1].y = b;
  z[L - 1 - n].x = -a;
  z[L - 1 - n].y = -b;
}

// One real row into the real (part 0) or imaginary (part 1) lane of an odd extension.
template <typename T>
__device__ __forceinline__ void put_one(typename C2<T>::t* z, int L, int n, T a, int part) {
  if (part) {
    z[n + 1].y = a;
    z[L - 1 - n].y = -a;
  } else {
    z[n + 1].x = a;
    z[L - 1 - n].x = -a;
  }
}

// Diagonal scaling data for pass Y (Sec. 3.2.1): A_w = 1/dt + lambda/(2 Re), lambda = (lx_k + ly_l)/h^2
// with lx_k = 4 sin^2(pi k/(2 Mx)).  Boundary-ring terms of a nested level enter as a rank-4 sum over the
// sine transforms of the four ring sides (left/right along y, bottom/top along x).  Tables and constants
// are in the precision of the pass (no double arithmetic per element in the FP32 path).
template <typename T>
struct SpecParams {
  const T* lx;   // [Mx] (index k = 1..Nx used)
  const T* ly;   // [My]
  const T* sx1;  // sin(pi k/Mx)
  const T* sxN;  // sin(pi k Nx/Mx)
  const T* sy1;
  const T* syN;
  const T* ring;  // 8 spectra: wL wR (len Ny) wB wT (len Nx) sL sR sB sT, each stride ring_ld; NULL = no ring
  long ring_ld;
  T inv_h2, inv_dt, inv_2re, norm;  // norm = 4/(Mx My)
  T ring_w;                         // inv_2re * inv_h2
  int Mx, My;
};

// The twiddle table for shared memory, held in registers between its load and its store (entries
// m = tid + q * blockDim.x, NQ >= L / blockDim.x of them per thread), so that a pass can load this constant
// table before it waits for its predecessor and store it once its own loads are in flight.  The table goes
// to shared memory when the launch gave the kernel room for it (dynamic shared memory of at least
// end_bytes, the table ending there); otherwise the stages read it from global memory.
template <typename T, int NQ>
struct TwiddleStage {
  using c2 = typename C2<T>::t;
  c2 v[NQ];
  bool on;
  __device__ __forceinline__ void load(const c2* __restrict__ tw, int L, size_t end_bytes) {
    unsigned dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    on = (size_t)dyn >= end_bytes;
    if (on) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int m = threadIdx.x + q * blockDim.x;
        if (m < L) v[q] = tw[m];
      }
    }
  }
  __device__ __forceinline__ const c2* store(c2* tws, const c2* tw, int L) const {
    if (!on) return tw;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int m = threadIdx.x + q * blockDim.x;
      if (m < L) tws[m] = v[q];
    }
    return tws;
  }
};

// Rows row and row + 1 of a transposed output at offset off (row + 1 next to row): the DST pair read off one
// complex transform z (row: -Im(z)/2, row + 1: Re(z)/2), one vector store when both rows exist and the
// address is aligned for it.
template <typename T>
__device__ __forceinline__ void store_pair(T* __restrict__ out, long off, int row, int nrows,
                                           typename C2<T>::t z) {
  using c2 = typename C2<T>::t;
  const T a = T(-0.5) * z.y, b = T(0.5) * z.x;
  T* p = out + off;
  if (row + 1 < nrows && (reinterpret_cast<uintptr_t>(p) & (sizeof(c2) - 1)) == 0) {
    c2 v;
    v.x = a;
    v.y = b;
    *reinterpret_cast<c2*>(p) = v;
  } else {
    if (row < nrows) p[0] = a;
    if (row + 1 < nrows) p[1] = b;
  }
}

// The passes below are bound by latency (a level is a few hundred kB and sits in L2), so each issues all
// the global loads of a pair of rows before its first shared-memory store: a thread owns the entries
// n = tid + m * blockDim.x, m < 2 PER, of every row of its CTA (N < L/2 <= 2 PER blockDim.x), and a pair of
// rows packed into one complex transform is read and written by the same thread.

// Pass XF: rows j of `in` (row stride in_ld, nrows rows of length N) -> unnormalised DST along the row ->
// transposed store out[k*out_ld + j] (k = 0..N-1).  blockIdx.y indexes a batch with element strides.
template <typename T, int PER, int R3 = 1>
__global__ void __launch_bounds__(256) k_xf(const T* __restrict__ in, long in_ld, long in_bs, int nrows, int N,
                                            T* __restrict__ out, long out_ld, long out_bs,
                                            const typename C2<T>::t* __restrict__ tw, int logL, int nf) {
  using c2 = typename C2<T>::t;
  constexpr int NC = 2 * PER * R3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2* buf = reinterpret_cast<c2*>(smem_raw);
  const int L = R3 << logL;  // logL: log2 of the power-of-two part of the length
  const int tid = threadIdx.x, nthr = blockDim.x;
  TwiddleStage<T, 4 * PER * R3> ts;
  ts.load(tw, L, ((size_t)nf + 1) * L * sizeof(c2));
  pdl_enter();
  const int row0 = blockIdx.x * 2 * nf;
  in += (long)blockIdx.y * in_bs;
  out += (long)blockIdx.y * out_bs;
  zero_ends<T>(buf, nf, L);
  for (int f = 0; f < nf; ++f) {
    const int r0 = row0 + 2 * f;
    T a[NC], b[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int n = tid + m * nthr;
      a[m] = (n < N && r0 < nrows) ? in[(long)r0 * in_ld + n] : T(0);
      b[m] = (n < N && r0 + 1 < nrows) ? in[(long)(r0 + 1) * in_ld + n] : T(0);
    }
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int n = tid + m * nthr;
      if (n < N) put_pair<T>(buf + (long)f * L, L, n, a[m], b[m]);
    }
  }
  const c2* tws = ts.store(buf + (long)nf * L, tw, L);
  __syncthreads();
  block_fft<T, PER, R3>(buf, L, logL, tws);
  const int lognf = __ffs(nf) - 1;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const int idx = tid + q * nthr;  // nf * N < 2 PER R3 blockDim.x
    if (idx < nf * N) {
      const int f = idx & (nf - 1), k = idx >> lognf;
      const int row = row0 + 2 * f;
      store_pair<T>(out, (long)k * out_ld + row, row, nrows, buf[(long)f * L + k + 1]);
    }
  }
}

// Per-row terms of the diagonal solve of pass Y at x-frequency k (1-based; rows beyond nrows are inactive).
// The boundary sine tables sx1, sxN, sy1, syN and the ring are read only when sp.ring is set (callers
// without a ring may leave them null).
template <typename T>
struct YRow {
  T lx, sx1, sxN, wb, wt, sb, st;  // wb..st: the bottom/top ring spectra of w and s at k
  bool on;
};

template <typename T>
__device__ __forceinline__ YRow<T> y_row(const SpecParams<T>& sp, int k, int nrows) {
  YRow<T> r;
  r.on = k <= nrows;
  const int kk = r.on ? k : 1;
  r.lx = sp.lx[kk];
  r.sx1 = r.sxN = r.wb = r.wt = r.sb = r.st = T(0);
  if (sp.ring) {  // the boundary sine tables exist only with a ring
    r.sx1 = sp.sx1[kk];
    r.sxN = sp.sxN[kk];
    r.wb = sp.ring[2 * sp.ring_ld + (kk - 1)];
    r.wt = sp.ring[3 * sp.ring_ld + (kk - 1)];
    r.sb = sp.ring[6 * sp.ring_ld + (kk - 1)];
    r.st = sp.ring[7 * sp.ring_ld + (kk - 1)];
  }
  return r;
}

// Pass Y: rows k of `in` (x-frequency k+1; nrows = Nx rows of length N = Ny) -> DST along y -> diagonal
// solve for w~ = (r^ + bc_w)/A_w and s~ = (w~ + bc_s)/lambda, both times norm -> DST along y (inverse) ->
// transposed stores outw[j*out_ld + k], outs[j*out_ld + k].  DEF: rows of `inr` (x-transforms of a defect d,
// same layout) are transformed beside `in` and enter the streamfunction only: s~ = (w~ + bc_s + d^)/lambda.
template <typename T, int PER, int R3 = 1, bool DEF = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_ysolve(const T* __restrict__ in, long in_ld, long in_bs, int nrows, int N,
                                                T* __restrict__ outw, T* __restrict__ outs, long out_ld,
                                                long out_bs, const typename C2<T>::t* __restrict__ tw, int logL,
                                                int nf, SpecParams<T> sp, const T* __restrict__ inr) {
  using c2 = typename C2<T>::t;
  constexpr int NC = 2 * PER * R3;
  constexpr int NB = DEF ? 2 : 1;  // forward transforms per row pair
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [2 nf][L]: the forward transforms of the row pairs of `in` (buffers 0..nf-1) and `inr` (nf..2nf-1), replaced
  // in place by the w~ (0..nf-1) and s~ (nf..2nf-1) spectra: a thread reads and writes the same frequencies
  // l + 1 <= N and writes the mirrored ones L - 1 - l >= L - N, which no thread reads
  c2* buf = reinterpret_cast<c2*>(smem_raw);
  const int L = R3 << logL;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int row0 = blockIdx.x * 2 * nf;
  // constant tables (set up with the context): loaded before the wait for the predecessor
  TwiddleStage<T, 4 * PER * R3> ts;
  ts.load(tw, L, (2 * (size_t)nf + 1) * L * sizeof(c2));
  pdl_enter();
  in += (long)blockIdx.y * in_bs;
  if (DEF) inr += (long)blockIdx.y * in_bs;
  outw += (long)blockIdx.y * out_bs;
  outs += (long)blockIdx.y * out_bs;
  const T* ring = sp.ring;
  zero_ends<T>(buf, NB * nf, L);
  for (int q = 0; q < NB * nf; ++q) {  // rows of `in` into buffers 0..nf-1, rows of `inr` into nf..2nf-1
    const int f = q < nf ? q : q - nf;
    const T* src = q < nf ? in : inr;
    const int r0 = row0 + 2 * f;
    T a[NC], b[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int n = tid + m * nthr;
      a[m] = (n < N && r0 < nrows) ? src[(long)r0 * in_ld + n] : T(0);
      b[m] = (n < N && r0 + 1 < nrows) ? src[(long)(r0 + 1) * in_ld + n] : T(0);
    }
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int n = tid + m * nthr;
      if (n < N) put_pair<T>(buf + (long)q * L, L, n, a[m], b[m]);
    }
  }
  const c2* tws = ts.store(buf + 2L * nf * L, tw, L);
  __syncthreads();
  block_fft<T, NB * PER, R3>(buf, L, logL, tws);
  // the per-column tables (eigenvalues, boundary sines, ring spectra) are read here, after the transforms,
  // rather than held in registers across them (more resident CTAs)
  for (int f = 0; f < nf; ++f) {
    const YRow<T> rw[2] = {y_row<T>(sp, row0 + 2 * f + 1, nrows), y_row<T>(sp, row0 + 2 * f + 2, nrows)};
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int l0 = tid + m * nthr;
      if (l0 >= N) continue;
      const T lyv = sp.ly[l0 + 1];
      T sy1v = T(0), syNv = T(0), rc[4] = {T(0), T(0), T(0), T(0)};  // left/right ring spectra of w and s
      if (ring) {
        sy1v = sp.sy1[l0 + 1];
        syNv = sp.syN[l0 + 1];
        rc[0] = ring[0 * sp.ring_ld + l0];
        rc[1] = ring[1 * sp.ring_ld + l0];
        rc[2] = ring[4 * sp.ring_ld + l0];
        rc[3] = ring[5 * sp.ring_ld + l0];
      }
      const c2 z = buf[(long)f * L + l0 + 1];
      c2 zd;
      if (DEF) zd = buf[(long)(nf + f) * L + l0 + 1];
      T wv[2], sv[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        T rh = e ? T(0.5) * z.x : T(-0.5) * z.y;
        if (rw[e].on) {
          const T lam = (rw[e].lx + lyv) * sp.inv_h2;
          const T aw = sp.inv_dt + lam * sp.inv_2re;
          T bcs = T(0);
          if (ring) {
            const T bw = rw[e].sx1 * rc[0] + rw[e].sxN * rc[1] + rw[e].wb * sy1v + rw[e].wt * syNv;
            bcs = rw[e].sx1 * rc[2] + rw[e].sxN * rc[3] + rw[e].sb * sy1v + rw[e].st * syNv;
            rh += bw * sp.ring_w;
            bcs *= sp.inv_h2;
          }
          const T wt = rh / aw;
          if (DEF) bcs += e ? T(0.5) * zd.x : T(-0.5) * zd.y;
          const T st = (wt + bcs) / lam;
          wv[e] = wt * sp.norm;
          sv[e] = st * sp.norm;
        } else {
          wv[e] = T(0);
          sv[e] = T(0);
        }
      }
      // the w~ rows of a pair share one complex transform (buffers 0..nf-1), the s~ rows another
      // (nf..2nf-1): s~ is smaller than w~ by ~1/lambda, so packing w~ with s~ would bury s~ in rounding.
      put_pair<T>(buf + (long)f * L, L, l0, wv[0], wv[1]);
      put_pair<T>(buf + (long)(nf + f) * L, L, l0, sv[0], sv[1]);
    }
  }
  __syncthreads();
  zero_ends<T>(buf, 2 * nf, L);  // the forward transforms left rounding at frequencies 0 and L/2
  __syncthreads();
  block_fft<T, 2 * PER, R3>(buf, L, logL, tws);
  const int lognf = __ffs(nf) - 1;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const int idx = tid + q * nthr;  // nf * N < 2 PER R3 blockDim.x
    if (idx < nf * N) {
      const int f = idx & (nf - 1), j = idx >> lognf;
      const int row = row0 + 2 * f;
      const long o = (long)j * out_ld + row;
      store_pair<T>(outw, o, row, nrows, buf[(long)f * L + j + 1]);
      store_pair<T>(outs, o, row, nrows, buf[(long)(nf + f) * L + j + 1]);
    }
  }
}

// Pass XI: rows j of inw and ins (length N = Nx) -> DST along x -> w, s rows written to the level fields
// (row j+1, columns 1..N of a vertex array of type TF with row stride f_ld).  mode 0: store, 1: subtract,
// 2: add (fields of type TF = double with float transforms: the increments of the mixed mode).
// blockIdx.x = 2 * (row block) + field: a CTA takes 2*nf rows of one field (0: w, 1: s), so w and s run on
// different CTAs (twice the CTAs, one transform buffer per row pair); rows j, j+1 share one FFT.
template <typename T, int PER, typename TF = T, int R3 = 1>
__global__ void __launch_bounds__(256) k_xi(const T* __restrict__ inw, const T* __restrict__ ins, long in_ld,
                                            long in_bs, int nrows, int N, TF* __restrict__ fw, TF* __restrict__ fs,
                                            long f_ld, long f_bs, int mode,
                                            const typename C2<T>::t* __restrict__ tw, int logL, int nf) {
  using c2 = typename C2<T>::t;
  constexpr int NC = 2 * PER * R3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2* buf = reinterpret_cast<c2*>(smem_raw);
  const int L = R3 << logL;
  const int tid = threadIdx.x, nthr = blockDim.x;
  TwiddleStage<T, 4 * PER * R3> ts;
  ts.load(tw, L, ((size_t)nf + 1) * L * sizeof(c2));
  pdl_enter();
  const int field = blockIdx.x & 1;
  const int row0 = (blockIdx.x >> 1) * 2 * nf;
  const T* in = (field ? ins : inw) + (long)blockIdx.y * in_bs;
  TF* fo = (field ? fs : fw) + (long)blockIdx.y * f_bs;
  // modes 1 and 2 update the field: the old values under the first pair of rows load with the inputs
  TF old[NC][2];
  if (mode != 0) {
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int i = tid + m * nthr;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const bool ok = i < N && row0 + e < nrows;
        old[m][e] = ok ? fo[(long)(row0 + e + 1) * f_ld + 1 + i] : TF(0);
      }
    }
  }
  zero_ends<T>(buf, nf, L);
  for (int f = 0; f < nf; ++f) {
    const int r0 = row0 + 2 * f;
    T a[NC], b[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int n = tid + m * nthr;
      a[m] = (n < N && r0 < nrows) ? in[(long)r0 * in_ld + n] : T(0);
      b[m] = (n < N && r0 + 1 < nrows) ? in[(long)(r0 + 1) * in_ld + n] : T(0);
    }
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int n = tid + m * nthr;
      if (n < N) put_pair<T>(buf + (long)f * L, L, n, a[m], b[m]);
    }
  }
  const c2* tws = ts.store(buf + (long)nf * L, tw, L);
  __syncthreads();
  block_fft<T, PER, R3>(buf, L, logL, tws);
  for (int f = 0; f < nf; ++f) {
#pragma unroll
    for (int m = 0; m < NC; ++m) {
      const int i = tid + m * nthr;
      if (i >= N) continue;
      const c2 z = buf[(long)f * L + i + 1];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int r = row0 + 2 * f + e;
        if (r >= nrows) continue;
        const long o = (long)(r + 1) * f_ld + 1 + i;
        const T v = e ? T(0.5) * z.x : T(-0.5) * z.y;
        if (mode == 0) {
          fo[o] = TF(v);
        } else {
          const TF prev = f == 0 ? old[m][e] : fo[o];
          fo[o] = mode == 1 ? prev - TF(v) : prev + TF(v);
        }
      }
    }
  }
}

// CTAs of pass XI for nrows rows: a row block per field.
inline unsigned xi_blocks(int nrows, int nf) { return 2u * (unsigned)((nrows + 2 * nf - 1) / (2 * nf)); }

}  // namespace dst
