"""Host-side check of the stage-ordered twiddle table of the shared-memory FFT (no GPU needed).

dst::block_fft reads, in a radix-4 stage with ns = 4^s > 1, the twiddle w_r(k) = exp(-2 pi i r k / (4 ns))
from entry (ns - 4) + (r - 1) ns + k of the table, and in the final radix-2 stage of an odd log2 L the
twiddle exp(-2 pi i k / L) from entry L/2 - 4 + k.  Every producer of the table stores, at entry p, the
exponent m = twiddle_exponent(p, log2 L).  This test compiles a small host program against the library's
own header and checks, for every transform length the library supports, that each entry the stages read
lies inside the table and holds the exponent of the radix-2 Stockham recursion: m = r k L / (4 ns) for the
radix-4 stages and m = k for the radix-2 stage.  It also checks that different (stage, r, k) never share an
entry unless they need the same twiddle.
"""

import os
import shutil
import subprocess

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(REPO, "paper_2103_06415_gb300", "csrc", "dst.cuh")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "@HEADER@"
void fsi_set_last_cuda_error(cudaError_t, const char*, const char*, int) {}
void fsi_set_last_message(const char*) {}
int main() {
  int bad = 0, checked = 0;
  for (int logL = 3; logL <= 13; ++logL) {
    const int L = 1 << logL;
    std::vector<int> owner(L, -1);  // exponent the stages expect at each entry (-1: unused)
    auto check = [&](int idx, int m_expect) {
      ++checked;
      if (idx < 0 || idx >= L) { ++bad; return; }
      if (dst::twiddle_exponent(idx, logL) != m_expect) ++bad;
      if (owner[idx] >= 0 && owner[idx] != m_expect) ++bad;
      owner[idx] = m_expect;
    };
    int rem = logL, logNs = 0;
    while (rem > 0) {  // the stage sequence of dst::block_fft
      if (rem >= 2) {
        if (logNs > 0)
          for (int k = 0; k < (1 << logNs); ++k)
            for (int r = 1; r < 4; ++r)
              check(((1 << logNs) - 4) + ((r - 1) << logNs) + k, r * k * (L / (4 << logNs)));
        logNs += 2;
        rem -= 2;
      } else {
        for (int k = 0; k < (1 << logNs); ++k) check((1 << (logL - 1)) - 4 + k, k);
        logNs += 1;
        rem -= 1;
      }
    }
  }
  printf("checked %d bad %d\n", checked, bad);
  return bad != 0 || checked == 0;
}
"""


def test_stage_order_twiddle_table_matches_stockham_exponents(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "twiddle_order.cu"
    src.write_text(PROGRAM.replace("@HEADER@", HEADER))
    exe = tmp_path / "twiddle_order"
    build = subprocess.run([nvcc, "-std=c++17", "-o", str(exe), str(src)], capture_output=True, text=True, timeout=300)
    assert build.returncode == 0, build.stderr[-2000:]
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "bad 0" in run.stdout
