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
// the result loses accuracy gradually but stays finite.  Checked on the GPU
// against FP64 references over dense argument sweeps of every tier
// (tests/test_fastmath_gpu.py): expi2_m1 within 2.5e-7 relative to |w| for
// |h| < 3000 (largest seen 2.14e-7, about 3.6 units of FP32 rounding of
// |w|), expm1_f within 1.5e-7 relative (largest seen 1.15e-7, at x near 17,
// where 2^k - 1 is not a float), the shear constants within 3e-7 of the
// exact rotation of a unit vector.
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
  if (fabsf(h) < 0.125f) {
    // Small half phases (the usual case for a stable time step): the series of
    // exp(2ih) - 1 directly, truncation below 1e-12 relative for |h| < 1/8:
    // cos 2h - 1 = -2h^2 + 2h^4/3 - 4h^6/45 + 2h^8/315,
    // sin 2h = 2h - 4h^3/3 + 4h^5/15 - 8h^7/315 + 4h^9/2835.
    const float h2 = h * h;
    wre = h2 * fmaf(h2, fmaf(h2, fmaf(h2, 6.3492063492e-3f, -8.8888888889e-2f), 0.66666666667f), -2.0f);
    wim = h * fmaf(h2, fmaf(h2, fmaf(h2, fmaf(h2, 1.4109347443e-3f, -2.5396825397e-2f), 0.26666666667f),
                            -1.3333333333f), 2.0f);
    return;
  }
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

// Shear constants of a rotation by 2h: t = tan(h), s = sin(2h); neg is set
// when the rotation is by 2r + pi with |r| <= pi/4 (apply R(2r), then negate).
// Series for small |h| (three tiers: |h| < 1/32, < 1/8, else reduced), so the
// common case of a small phase costs a handful of fma:
// tan h = h + h^3/3 + 2h^5/15 + 17h^7/315 + 62h^9/2835 + ...,
// sin 2h = 2h - 4h^3/3 + 4h^5/15 - 8h^7/315 + 4h^9/2835 - ...
// The general tiers live out of line: kernels inline only the warp-uniform
// small-phase series, and a single copy of this routine serves the rare
// warps with larger phases (keeps the row pass within the instruction cache).
struct ShearConsts {
  float t, s;
  int neg;
};
static __device__ __noinline__ ShearConsts shear_consts_2h_general(float h);

__device__ __forceinline__ void shear_consts_2h(float h, float &t, float &s, bool &neg) {
  const ShearConsts r = shear_consts_2h_general(h);
  t = r.t;
  s = r.s;
  neg = r.neg != 0;
}

static __device__ __noinline__ ShearConsts shear_consts_2h_general(float h) {
  float t, s;
  bool neg;
  const float ah = fabsf(h);
  neg = false;
  if (ah < 0.03125f) {  // truncation below 2e-11 relative
    const float h2 = h * h;
    t = h * fmaf(h2, fmaf(h2, 0.13333333333f, 0.33333333333f), 1.0f);
    s = h * fmaf(h2, fmaf(h2, 0.26666666667f, -1.3333333333f), 2.0f);
  } else if (ah < 0.125f) {  // truncation below 1e-12 relative
    const float h2 = h * h;
    t = h * fmaf(h2, fmaf(h2, fmaf(h2, fmaf(h2, 2.1869488536e-2f, 5.3968253968e-2f), 0.13333333333f),
                      0.33333333333f), 1.0f);
    s = h * fmaf(h2, fmaf(h2, fmaf(h2, fmaf(h2, 1.4109347443e-3f, -2.5396825397e-2f), 0.26666666667f),
                      -1.3333333333f), 2.0f);
  } else {
    const int n = __float2int_rn(h * kTwoOverPi);
    const float fn = (float)n;
    float r = fmaf(-fn, kPio2A, h);
    r = fmaf(-fn, kPio2B, r);
    r = fmaf(-fn, kPio2C, r);
    const float r2 = r * r;
    float ps = fmaf(r2, 2.7557319224e-6f, -1.9841269841e-4f);
    ps = fmaf(r2, ps, 8.3333333333e-3f);
    ps = fmaf(r2, ps, -1.6666666667e-1f);
    const float sr = fmaf(r * r2, ps, r);
    float pc = fmaf(r2, -2.7557319224e-7f, 2.4801587302e-5f);
    pc = fmaf(r2, pc, -1.3888888889e-3f);
    pc = fmaf(r2, pc, 4.1666666667e-2f);
    pc = fmaf(r2, pc, -0.5f);
    const float cr = fmaf(r2, pc, 1.0f);
    t = sr / cr;
    s = 2.0f * sr * cr;
    neg = (n & 1) != 0;  // exp(2ih) = -exp(2ir)
  }
  return ShearConsts{t, s, neg ? 1 : 0};
}

// Cubic series, for callers that know |h| < 1/64 for a whole warp: the first
// omitted terms (2h^5/15 and 4h^5/15) are below 8e-9 relative to t and s.
__device__ __forceinline__ void shear_consts_2h_tiny(float h, float &t, float &s) {
  const float h2 = h * h;
  t = h * fmaf(h2, 0.33333333333f, 1.0f);
  s = h * fmaf(h2, -1.3333333333f, 2.0f);
}

// The middle tier alone, for callers that know |h| < 1/8 for a whole warp.
__device__ __forceinline__ void shear_consts_2h_small(float h, float &t, float &s) {
  const float h2 = h * h;
  t = h * fmaf(h2, fmaf(h2, fmaf(h2, fmaf(h2, 2.1869488536e-2f, 5.3968253968e-2f), 0.13333333333f),
                    0.33333333333f), 1.0f);
  s = h * fmaf(h2, fmaf(h2, fmaf(h2, fmaf(h2, 1.4109347443e-3f, -2.5396825397e-2f), 0.26666666667f),
                    -1.3333333333f), 2.0f);
}

// Double precision: the CUDA math library.
__device__ __forceinline__ void shear_consts_2h(double h, double &t, double &s, bool &neg) {
  double sh, ch;
  sincos(h, &sh, &ch);
  const double a = fabs(h);
  neg = false;
  if (a <= 0.78539816339744830962) {
    t = sh / ch;
    s = 2.0 * sh * ch;
  } else {
    // rotate by 2h - pi (|h - pi/2| < pi/2 folded to |r| <= pi/4) and negate
    const double n = rint(h * 0.63661977236758134308);
    const double r = h - n * 1.57079632679489661923;
    double sr, cr;
    sincos(r, &sr, &cr);
    t = sr / cr;
    s = 2.0 * sr * cr;
    neg = (((long long)n) & 1) != 0;
  }
}
__device__ __forceinline__ void shear_consts_2h_small(double h, double &t, double &s) {
  bool neg;
  shear_consts_2h(h, t, s, neg);
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
  if (fabsf(x) < 0.0625f) {
    // small arguments: x + x^2/2! + ... + x^7/7! (truncation below 1e-13 relative)
    float p = fmaf(x, 1.9841269841e-4f, 1.3888888889e-3f);
    p = fmaf(x, p, 8.3333333333e-3f);
    p = fmaf(x, p, 4.1666666667e-2f);
    p = fmaf(x, p, 1.6666666667e-1f);
    p = fmaf(x, p, 0.5f);
    return fmaf(x * x, p, x);
  }
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

// expm1 for |x| < 1/2 (callers that know the bound for a whole warp):
// Taylor series to x^11/11!, truncation below 1e-12 relative.
__device__ __forceinline__ float expm1_small(float x) {
  float p = fmaf(x, 2.5052108385e-8f, 2.7557319224e-7f);
  p = fmaf(x, p, 2.7557319224e-6f);
  p = fmaf(x, p, 2.4801587302e-5f);
  p = fmaf(x, p, 1.9841269841e-4f);
  p = fmaf(x, p, 1.3888888889e-3f);
  p = fmaf(x, p, 8.3333333333e-3f);
  p = fmaf(x, p, 4.1666666667e-2f);
  p = fmaf(x, p, 1.6666666667e-1f);
  p = fmaf(x, p, 0.5f);
  return fmaf(x * x, p, x);
}

// expm1 for |x| < 1/4 (callers that know the bound for a whole warp):
// Taylor series to x^6/6!.  The first omitted term bounds the truncation by
// |x|^6/7! relative, 4.8e-8 at the edge, below half a unit of FP32 rounding.
__device__ __forceinline__ float expm1_quarter(float x) {
  float p = fmaf(x, 1.3888888889e-3f, 8.3333333333e-3f);
  p = fmaf(x, p, 4.1666666667e-2f);
  p = fmaf(x, p, 1.6666666667e-1f);
  p = fmaf(x, p, 0.5f);
  return fmaf(x * x, p, x);
}

// Double precision: the CUDA math library.
__device__ __forceinline__ double expm1_small(double x) { return expm1(x); }
__device__ __forceinline__ double expm1_quarter(double x) { return expm1(x); }
__device__ __forceinline__ void expi2_m1(double h, double &wre, double &wim) {
  double s, c;
  sincos(h, &s, &c);
  wre = -2.0 * s * s;
  wim = 2.0 * s * c;
}
__device__ __forceinline__ double expm1_f(double x) { return expm1(x); }

}  // namespace spgpe
