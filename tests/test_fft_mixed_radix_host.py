"""Host-side check of the shared-memory FFT stages for every transform length the library takes (no GPU).

The passes transform rows of length L = 2(N + 1) for grids of N + 1 = 2^k or 3 * 2^k cells per axis, so
L = R3 * 2^logP with R3 = 1 or 3.  dst::block_fft runs radix-4 stages (one radix-2 stage for an odd logP) and,
for R3 = 3, a final radix-3 stage; each stage is a load of every butterfly's inputs, a barrier, and a
compute-and-store.  The stage functions are host-callable, so this test compiles a host program against the
library's own header that runs them exactly as block_fft does -- the same launch shape (threads, PER, the
number nf of transforms per CTA), the same butterfly numbering b = tid + q * threads, every load of a stage
before its stores -- over a buffer with guard zones on both sides, and checks for every length:

* the result equals a direct DFT (long double sums) to rounding: relative max error < 1e-13 in double,
  < 1e-5 in float, for each of the nf transforms of the CTA;
* the guard zones are untouched (no store outside the CTA's nf * L entries) and no stage reads a guard value
  (guards hold NaN, which would reach the result);
* every table entry a stage reads holds the exponent it needs (the table built by twiddle_exponent).
"""

import os
import shutil
import subprocess

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(REPO, "paper_2103_06415_gb300", "csrc", "dst.cuh")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include <vector>
#include "@HEADER@"
void fsi_set_last_cuda_error(cudaError_t, const char*, const char*, int) {}
void fsi_set_last_message(const char*) {}

template <typename T, int R3>
double run(int logP, int PER, int nthr, int nf) {
  using c2 = typename C2<T>::t;
  const int L = R3 << logP;
  std::vector<c2> tw(L);
  for (int p = 0; p < L; ++p) {
    const long double a = -2.0L * 3.14159265358979323846264338327950288L * dst::twiddle_exponent(p, logP, R3) / L;
    tw[p].x = (T)cosl(a);
    tw[p].y = (T)sinl(a);
  }
  const long n = (long)nf * L;
  std::vector<c2> all(n + 2 * L);
  const T nan = (T)NAN;
  for (auto& z : all) { z.x = nan; z.y = nan; }
  c2* buf = all.data() + L;
  std::vector<c2> x0(n);
  unsigned s = 12345u + L;
  for (long i = 0; i < n; ++i) {
    s = s * 1664525u + 1013904223u; x0[i].x = (T)((s >> 8) * (1.0 / 16777216.0) - 0.5);
    s = s * 1664525u + 1013904223u; x0[i].y = (T)((s >> 8) * (1.0 / 16777216.0) - 0.5);
    buf[i] = x0[i];
  }
  // block_fft, thread by thread within each phase
  std::vector<c2> v((size_t)nthr * 12 * PER);
  int logNs = 0, rem = logP;
  while (rem > 0) {
    if (rem >= 2) {
      for (int tid = 0; tid < nthr; ++tid)
        for (int q = 0; q < PER * R3; ++q) dst::r4_load<T, R3>(buf, L, logP, tid + q * nthr, &v[(size_t)tid * 12 * PER + 4 * q]);
      for (int tid = 0; tid < nthr; ++tid)
        for (int q = 0; q < PER * R3; ++q)
          dst::r4_store<T, R3>(buf, L, logP, logNs, tid + q * nthr, tw.data(), &v[(size_t)tid * 12 * PER + 4 * q]);
      logNs += 2; rem -= 2;
    } else {
      for (int tid = 0; tid < nthr; ++tid)
        for (int q = 0; q < 2 * PER * R3; ++q) dst::r2_load<T, R3>(buf, L, logP, tid + q * nthr, &v[(size_t)tid * 12 * PER + 2 * q]);
      for (int tid = 0; tid < nthr; ++tid)
        for (int q = 0; q < 2 * PER * R3; ++q)
          dst::r2_store<T, R3>(buf, L, logP, logNs, tid + q * nthr, tw.data(), &v[(size_t)tid * 12 * PER + 2 * q]);
      logNs += 1; rem -= 1;
    }
  }
  if (R3 == 3) {
    for (int tid = 0; tid < nthr; ++tid)
      for (int q = 0; q < 4 * PER; ++q) dst::r3_load<T>(buf, L, logP, tid + q * nthr, &v[(size_t)tid * 12 * PER + 3 * q]);
    for (int tid = 0; tid < nthr; ++tid)
      for (int q = 0; q < 4 * PER; ++q) dst::r3_store<T>(buf, L, logP, tid + q * nthr, tw.data(), &v[(size_t)tid * 12 * PER + 3 * q]);
  }
  for (long i = 0; i < L; ++i) {  // guard zones untouched
    if (!std::isnan((double)all[i].x) || !std::isnan((double)all[n + L + i].x)) return 1e30;
  }
  double worst = 0.0;
  for (int f = 0; f < nf; ++f) {  // direct DFT of each transform
    double mx = 0.0, err = 0.0;
    for (int k = 0; k < L; ++k) {
      long double re = 0.0L, im = 0.0L;
      for (int j = 0; j < L; ++j) {
        const long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)(((long)j * k) % L) / L;
        const long double c = cosl(a), sn = sinl(a);
        re += x0[(long)f * L + j].x * c - x0[(long)f * L + j].y * sn;
        im += x0[(long)f * L + j].x * sn + x0[(long)f * L + j].y * c;
      }
      const c2 z = buf[(long)f * L + k];
      if (std::isnan((double)z.x) || std::isnan((double)z.y)) return 1e30;
      err = fmax(err, fmax(fabs((double)(z.x - re)), fabs((double)(z.y - im))));
      mx = fmax(mx, fmax(fabs((double)re), fabs((double)im)));
    }
    worst = fmax(worst, err / mx);
  }
  return worst;
}

int main() {
  int bad = 0, cases = 0;
  for (int R3 = 1; R3 <= 3; R3 += 2)
    for (int logP = 4; logP <= 12; ++logP) {
      const int P = 1 << logP;
      if (R3 * P > 4096) continue;  // grids up to 2048 cells per axis
      int nthr = P / 4;  // the passes' launch shape (fft_cfg)
      if (nthr < 32) nthr = 32;
      if (nthr > 256) nthr = 256;
      int per = 1;
      while (4 * per * nthr < P) per *= 2;
      const int nf = 4 * per * nthr / P;
      double ed, ef;
      if (R3 == 1) {
        ed = per == 1 ? run<double, 1>(logP, 1, nthr, nf) : per == 2 ? run<double, 1>(logP, 2, nthr, nf) : run<double, 1>(logP, 4, nthr, nf);
        ef = per == 1 ? run<float, 1>(logP, 1, nthr, nf) : per == 2 ? run<float, 1>(logP, 2, nthr, nf) : run<float, 1>(logP, 4, nthr, nf);
      } else {
        ed = per == 1 ? run<double, 3>(logP, 1, nthr, nf) : per == 2 ? run<double, 3>(logP, 2, nthr, nf) : run<double, 3>(logP, 4, nthr, nf);
        ef = per == 1 ? run<float, 3>(logP, 1, nthr, nf) : per == 2 ? run<float, 3>(logP, 2, nthr, nf) : run<float, 3>(logP, 4, nthr, nf);
      }
      ++cases;
      const bool ok = ed < 1e-13 && ef < 1e-5;
      if (!ok) ++bad;
      printf("L %5d  nthr %3d per %d nf %d  double %.2e  float %.2e  %s\n", R3 * P, nthr, per, nf, ed, ef, ok ? "ok" : "BAD");
    }
  printf("cases %d bad %d\n", cases, bad);
  return bad != 0 || cases == 0;
}
"""


def test_mixed_radix_fft_stages_match_direct_dft(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "fft_stages.cu"
    src.write_text(PROGRAM.replace("@HEADER@", HEADER))
    exe = tmp_path / "fft_stages"
    build = subprocess.run([nvcc, "-std=c++17", "-O2", "-o", str(exe), str(src)], capture_output=True, text=True,
                           timeout=300)
    assert build.returncode == 0, build.stderr[-2000:]
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "bad 0" in run.stdout
