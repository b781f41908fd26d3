// Host-side stage twiddle tables of the block FFT plans (Plan in
// fft_core.cuh), computed in FP64 and rounded once to the working precision
// when uploaded.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

namespace spgpe {

// Twiddle table of the block FFT plan for n = 2^logn points with 2^loge
// values per thread (the plan of fft_core.cuh: S = max(ceil(logn / loge),
// ceil(logn / 4)) stages, radix bits split as evenly as possible, larger
// first).  Stage s >= 1 holds
// entries [r - 1][k], r = 1..R-1, k = 0..NS-1, for the root exp(-2 pi i m / n),
// m = r k n / (NS R); 16 bytes per entry:
//   complex64:  (tan(phi/2), sin(phi), g, g) with exp(-2 pi i m / n) = g e^{i phi},
//               g = +-1, phi in [-pi/2, pi/2] (three-shear rotation, exact sign);
//   complex128: (cos, -sin) of 2 pi m / n.
inline std::vector<double> stage_twiddles(int logn, int loge, bool single) {
  const double kTwoPi = 6.28318530717958647692528676655900577;
  const int n = 1 << logn;
  const int S = std::max((logn + loge - 1) / loge, (logn + 3) / 4);
  std::vector<double> out;
  int ns = 1;
  for (int s = 0; s < S; ++s) {
    const int bits = logn / S + (s < logn % S ? 1 : 0), R = 1 << bits;
    if (s > 0) {
      for (int r = 1; r < R; ++r)
        for (int k = 0; k < ns; ++k) {
          const long m = (long)r * k * (n / (ns * R));
          if (single) {
            double th = -kTwoPi * (double)m / n;      // (-2 pi, 0]
            if (th <= -0.5 * kTwoPi) th += kTwoPi;    // (-pi, pi]
            double g = 1.0, phi = th;
            if (std::fabs(th) > 0.25 * kTwoPi) {      // left half plane: rotate by th -+ pi, negate
              g = -1.0;
              phi = th > 0 ? th - 0.5 * kTwoPi : th + 0.5 * kTwoPi;
            }
            out.insert(out.end(), {std::tan(0.5 * phi), std::sin(phi), g, g});
          } else {
            out.insert(out.end(), {std::cos(kTwoPi * (double)m / n), -std::sin(kTwoPi * (double)m / n)});
          }
        }
    }
    ns *= R;
  }
  if (out.empty()) out.assign(single ? 4 : 2, 0.0);  // one-stage plans read no twiddle
  return out;
}

}  // namespace spgpe
