"""The host twiddle tables against the device FFT plans, on the CPU.

The device transform reads stage s's entry (r, k) at Plan::off(s) + (r-1) NS + k
with compile-time offsets; the host builds the table separately.  A small
program compiled against both (fft_core.cuh's Plan, twiddles.h's builder)
checks, for every plan the library can use (8 to 4096 points, 4 to 32 values
per thread, both precisions), that the table has exactly Plan::entries()
entries and that every entry decodes to the root the plan expects at that
position: exp(-2 pi i r k / (NS R)), from the DFT's definition.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2010_15069_gb300", "csrc")

CHECK = r"""
#include <cmath>
#include <complex>
#include <cstdio>
#include <utility>
#include "fft_core.cuh"
#include "twiddles.h"
using namespace spgpe;

template <int LOGN, int LOGE> int check() {
  using P = Plan<LOGN, LOGE>;
  int bad = 0;
  for (int single = 0; single < 2; ++single) {
    const std::vector<double> w = stage_twiddles(LOGN, LOGE, single);
    const int per = single ? 4 : 2;
    const size_t want = P::entries() > 0 ? P::entries() : 1;
    if (w.size() != want * per) {
      printf("size logn=%d loge=%d single=%d: %zu != %zu\n", LOGN, LOGE, single, w.size() / per, want);
      ++bad;
      continue;
    }
    for (int s = 1; s < P::S; ++s) {
      const int R = 1 << P::bits(s), NS = 1 << P::nsbits(s);
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < NS; ++k) {
          const double *e = &w[(size_t)(P::off(s) + (r - 1) * NS + k) * per];
          std::complex<double> got;
          if (single) {
            const double phi = 2.0 * std::atan(e[0]);
            if (std::fabs(std::sin(phi) - e[1]) > 1e-14 || std::fabs(e[2]) != 1.0 || e[3] != e[2]) ++bad;
            got = e[2] * std::complex<double>(std::cos(phi), std::sin(phi));
          } else {
            got = std::complex<double>(e[0], e[1]);
          }
          const double a = -2.0 * 3.14159265358979323846 * r * k / (double)(NS * R);
          if (std::abs(got - std::complex<double>(std::cos(a), std::sin(a))) > 1e-14) {
            if (bad < 10) printf("root logn=%d loge=%d single=%d s=%d r=%d k=%d\n", LOGN, LOGE, single, s, r, k);
            ++bad;
          }
        }
    }
  }
  return bad;
}

template <int LOGE, int... L> int all(std::integer_sequence<int, L...>) { return (check<L + 3, LOGE>() + ...); }

int main() {
  const int bad = all<2>(std::make_integer_sequence<int, 10>{}) + all<3>(std::make_integer_sequence<int, 10>{}) +
                  all<4>(std::make_integer_sequence<int, 10>{}) + all<5>(std::make_integer_sequence<int, 10>{});
  printf("%d mismatches\n", bad);
  return bad != 0;
}
"""


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_host_twiddle_tables_match_the_device_plans(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "check.cu"
    src.write_text(CHECK)
    exe = tmp_path / "check"
    r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                        str(src), "-o", str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "0 mismatches" in r.stdout
