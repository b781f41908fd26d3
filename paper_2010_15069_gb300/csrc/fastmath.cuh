// Elementary functions for the pointwise operators, written from their
// Taylor series with Cody-Waite range reduction (W. J. Cody and W. Waite,
// "Software Manual for the Elementary Functions", 1980): the argument is
// reduced by an integer multiple of a constant split into a leading part with
// trailing zero bits and a small correction, so the reduction is exact for
// the argument range used here.  Single precision only; the double-precision
// path calls the CUDA math library.
//
// They have no slow path: the reduction is exact for |h| < 2^12 pi/2 (phases
// of one substep far beyond anything a stable time step produces); beyond that
// the result loses accuracy gradually but stays finite.  Checked against FP64
// references: expi2_m1 within 2e-7 relative to |w| for |h| < 3000, expm1_f
// within 1e-7 relative.
#pragma once
#include <cuda_runtime.h>

namespace spgpe {

// pi/2 = A + B + C: A and B carry 12 significant bits each, so n*A and n*B
// are exact for |n| < 2^12; C is the rounded remainder.
constexpr float kPio2A = 1.57080078125f;             // 0x3FC91000
constexpr float kPio2B = -4.4535845518e-06f;         // 0xB6957000
constexpr float kPio2C = -8.7055163078e-10f;
constexpr float kTwoOverPi = 0.63661977236758134308f;

// w = exp(2 i h) - 1, to full relative precision of w, for the half phase h.
// With h = n pi/2 + r, |r| <= pi/4: exp(2ih) = (-1)^n exp(2ir) and
// exp(2ir) - 1 = -2 sin^2 r + 2i sin r cos r, sin r and cos r from their
// Taylor series (truncation below 2e-9 at |r| = pi/4).
__device__ __forceinline__ void expi2_m1(float h, float &wre, float &wim) {
  const int n = __float2int_rn(h * kTwoOverPi);
  const float fn = (float)n;
  float r = fmaf(-fn, kPio2A, h);
  r = fmaf(-fn, kPio2B, r);
  r = fmaf(-fn, kPio2C, r);
  const float r2 = r * r;
  // sin r = r (1 - r^2/3! + r^4/5! - r^6/7! + r^8/9!)
  float ps = fmaf(r2, 2.7557319224e-6f, -1.9841269841e-4f);
  ps = fmaf(r2, ps, 8.3333333333e-3f);
  ps = fmaf(r2, ps, -1.6666666667e-1f);
  const float sr = fmaf(r * r2, ps, r);
  // cos r = 1 - r^2/2! + r^4/4! - r^6/6! + r^8/8! - r^10/10!
  float pc = fmaf(r2, -2.7557319224e-7f, 2.4801587302e-5f);
  pc = fmaf(r2, pc, -1.3888888889e-3f);
  pc = fmaf(r2, pc, 4.1666666667e-2f);
  pc = fmaf(r2, pc, -0.5f);
  const float cr = fmaf(r2, pc, 1.0f);
  float a = -2.0f * sr * sr, b = 2.0f * sr * cr;
  if (n & 1) {  // exp(2ih) = -exp(2ir): w = -(1 + w') - 1
    a = -a - 2.0f;
    b = -b;
  }
  wre = a;
  wim = b;
}

// ln 2 = A + B, A with 12 significant bits (k * A exact for |k| < 2^12).
constexpr float kLn2A = 0.693115234375f;             // 0x3F317000
constexpr float kLn2B = 3.1946183299e-05f;
constexpr float kInvLn2 = 1.4426950408889634074f;

// exp(x) - 1 to full relative precision near 0.  x = k ln2 + r, |r| <= ln2/2,
// expm1(r) from its Taylor series to r^9/9! (truncation below 1e-11 relative),
// expm1(x) = 2^k expm1(r) + (2^k - 1).  Saturates to -1 below x = -87 and to
// about 1.7e38 above 88.
__device__ __forceinline__ float expm1_f(float x) {
  x = fminf(fmaxf(x, -87.0f), 88.0f);
  const int k = __float2int_rn(x * kInvLn2);
  const float fk = (float)k;
  float r = fmaf(-fk, kLn2A, x);
  r = fmaf(-fk, kLn2B, r);
  float p = fmaf(r, 2.7557319224e-6f, 2.4801587302e-5f);
  p = fmaf(r, p, 1.9841269841e-4f);
  p = fmaf(r, p, 1.3888888889e-3f);
  p = fmaf(r, p, 8.3333333333e-3f);
  p = fmaf(r, p, 4.1666666667e-2f);
  p = fmaf(r, p, 1.6666666667e-1f);
  p = fmaf(r, p, 0.5f);
  const float em = fmaf(r * r, p, r);
  if (k == 0) return em;
  const float s = __int_as_float((k + 127) << 23);  // 2^k, k in [-126, 127]
  return fmaf(s, em, s - 1.0f);
}

// Double precision: the CUDA math library.
__device__ __forceinline__ void expi2_m1(double h, double &wre, double &wim) {
  double s, c;
  sincos(h, &s, &c);
  wre = -2.0 * s * s;
  wim = 2.0 * s * c;
}
__device__ __forceinline__ double expm1_f(double x) { return expm1(x); }

}  // namespace spgpe
