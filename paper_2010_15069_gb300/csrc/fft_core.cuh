// Block-level Stockham FFT held in registers, exchanged through shared memory.
//
// Each thread of a length-N transform owns E = 2^LOGE elements of one
// sequence, at positions t + m*(N/E), m = 0..E-1, where t is the thread's
// index within the sequence.  A Stockham stage of radix R (R divides E) lets
// every thread run E/R butterflies; butterfly jv = t + b*(N/E) reads positions
// jv + r*N/R (which are again of the form t + m*N/E, m = b + r*E/R), applies
// the twiddles W_{Ns R}^{r (jv mod Ns)}, runs an R-point DFT in registers and
// writes position (jv / Ns)*Ns*R + (jv mod Ns) + r*Ns.  The output of the
// last stage lands on the positions the thread already holds, so a forward
// transform, a pointwise operator and an inverse transform can follow one
// another in registers with no shared-memory round trip in between; only the
// S-1 inner stage boundaries of each transform go through shared memory.
//
// Radix plan: S = max(ceil(LOGN / LOGE), ceil(LOGN / 4)) stages (radices of
// at most 16), log2 radices split as evenly as possible (2048 = 16*16*8 at
// E = 16, 256 = 16*16, 64 = 8*8, 512 = 8*8*8 at E = 32, ...).
#pragma once
#include <cuda_runtime.h>

namespace spgpe {

template <class T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <class T> __device__ __forceinline__ T d_fma(T a, T b, T c) {
  if constexpr (sizeof(T) == 4) return fmaf(a, b, c); else return fma(a, b, c);
}
template <class T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
// Single precision: one packed add of the (re, im) pair (sm_100 family
// f32x2 arithmetic; each lane rounds exactly as the scalar add does).
template <> __device__ __forceinline__ cx<float> cadd(cx<float> a, cx<float> b) {
  const float2 r = __fadd2_rn(make_float2(a.re, a.im), make_float2(b.re, b.im));
  return {r.x, r.y};
}
template <> __device__ __forceinline__ cx<float> csub(cx<float> a, cx<float> b) {
  const float2 r = __fadd2_rn(make_float2(a.re, a.im), make_float2(-b.re, -b.im));
  return {r.x, r.y};
}
template <class T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.re * s, a.im * s}; }
template <class T> __device__ __forceinline__ T cabs2(cx<T> a) { return a.re * a.re + a.im * a.im; }

// Rotation of a by the angle phi with tan(phi/2) = t and sin(phi) = s, as
// three shears (x -= t y; y += s x; x -= t y).  Each shear has determinant
// one whatever the rounding of t and s, so the rotation never scales |a|
// systematically; a rounded (cos, sin) pair would scale it by a fixed factor
// 1 + O(2^-24) at every use, which accumulates over thousands of transforms.
template <class T> __device__ __forceinline__ cx<T> shear_rot(cx<T> a, T t, T s) {
  const T x1 = d_fma(-t, a.im, a.re);
  const T y1 = d_fma(s, x1, a.im);
  return {d_fma(-t, y1, x1), y1};
}

// a * exp(SIGN * 2 pi i M / 16) for a compile-time M in [0, 8): quarter turns
// are exact (swap and negate), the rest is a three-shear rotation by +-pi/8 or
// +-pi/4.  Constants: tan(pi/16), sin(pi/8), tan(pi/8), sin(pi/4) to 20 digits,
// rounded once to T.
template <int SIGN, int M, class T>
__device__ __forceinline__ cx<T> w16(cx<T> a) {
  const T t16 = T(0.19891236737965800691), s8 = T(0.38268343236508977173);
  const T t8 = T(0.41421356237309504880), s4 = T(0.70710678118654752440);
  const T sg = T(SIGN);
  auto qturn = [&](cx<T> b) { return cx<T>{-sg * b.im, sg * b.re}; };  // * SIGN i
  if constexpr (M == 0) {
    return a;
  } else if constexpr (M == 1) {
    return shear_rot(a, sg * t16, sg * s8);
  } else if constexpr (M == 2) {
    return shear_rot(a, sg * t8, sg * s4);
  } else if constexpr (M == 3) {
    return qturn(shear_rot(a, -sg * t16, -sg * s8));
  } else if constexpr (M == 4) {
    return qturn(a);
  } else if constexpr (M == 5) {
    return qturn(shear_rot(a, sg * t16, sg * s8));
  } else if constexpr (M == 6) {
    return qturn(shear_rot(a, sg * t8, sg * s4));
  } else {
    const cx<T> b = shear_rot(a, -sg * t16, -sg * s8);
    return {-b.re, -b.im};
  }
}

// Stage twiddles, one table per transform plan, laid out per stage as
// [r - 1][k] (r = 1..R-1 the butterfly input, k = 0..NS-1 its position within
// the previous span), so that the threads of a warp read consecutive entries
// and every read has a compile-time offset; entry (r, k) of a stage is the
// forward root exp(-2 pi i m / N) with m = r k N / (NS R).
// Double precision: the root as a complex pair.  Single precision: the root
// is g R(phi) with g = +-1 and R(phi) a rotation by phi in [-pi/2, pi/2],
// stored as (tan(phi/2), sin(phi), g, g) and applied with three shears and a
// multiplication by g (one packed multiplication of the (re, im) pair by the
// (g, g) half of the entry).  A single-precision (cos, sin) pair is off unit modulus
// by about 2^-25 in a direction that does not average out over the set of
// roots; every element passes through these factors in every transform, and
// rounded pairs drain the norm by about 1e-7 per forward/inverse round trip.
template <class T> struct TwType;
template <> struct TwType<float> { using type = float4; };
template <> struct TwType<double> { using type = cx<double>; };

template <int SIGN, class T>
__device__ __forceinline__ cx<T> twiddle(cx<T> u, const typename TwType<T>::type &w) {
  if constexpr (sizeof(T) == 4) {
    const float t = SIGN < 0 ? w.x : -w.x, s = SIGN < 0 ? w.y : -w.y;  // inverse: R(-phi)
    const cx<T> r = shear_rot(u, t, s);
    const float2 gr = __fmul2_rn(make_float2(r.re, r.im), make_float2(w.z, w.w));  // (g, g)
    return {gr.x, gr.y};
  } else {
    const cx<T> c = SIGN < 0 ? w : cx<T>{w.re, -w.im};
    return cmul(u, c);
  }
}

template <int R>
__host__ __device__ constexpr int bitrev(int k) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) {
    r = (r << 1) | (k & 1);
    k >>= 1;
  }
  return r;
}

// One radix-2 decimation-in-frequency level of span LEN over an R-register
// array; twiddles W_LEN^k = W_16^(k*16/LEN).
template <int R, int LEN, int K, int SIGN, class T>
__device__ __forceinline__ void dif_bfly(cx<T> (&v)[R], int i) {
  if constexpr (K < LEN / 2) {
    const cx<T> a = v[i + K], b = v[i + K + LEN / 2];
    v[i + K] = cadd(a, b);
    v[i + K + LEN / 2] = w16<SIGN, K * (16 / LEN)>(csub(a, b));
    dif_bfly<R, LEN, K + 1, SIGN>(v, i);
  }
}

template <int R, int LEN, int SIGN, class T>
__device__ __forceinline__ void dif_level(cx<T> (&v)[R]) {
  if constexpr (LEN >= 2) {
#pragma unroll
    for (int i = 0; i < R; i += LEN) dif_bfly<R, LEN, 0, SIGN>(v, i);
    dif_level<R, LEN / 2, SIGN>(v);
  }
}

// In-register R-point DFT (R <= 16), natural order in and out:
// v_k <- sum_j v_j exp(SIGN 2 pi i j k / R).
template <int R, int SIGN, class T>
__device__ __forceinline__ void dft(cx<T> (&v)[R]) {
  static_assert(R >= 1 && R <= 16 && (R & (R - 1)) == 0, "radix must be 1..16, power of 2");
  dif_level<R, R, SIGN>(v);
  cx<T> t[R];
#pragma unroll
  for (int k = 0; k < R; ++k) t[k] = v[bitrev<R>(k)];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = t[k];
}

// Stage plan of a 2^LOGN transform with 2^LOGE elements per thread.
template <int LOGN, int LOGE>
struct Plan {
  static constexpr int S = (LOGN + LOGE - 1) / LOGE > (LOGN + 3) / 4 ? (LOGN + LOGE - 1) / LOGE : (LOGN + 3) / 4;
  __host__ __device__ static constexpr int bits(int s) { return LOGN / S + (s < LOGN % S ? 1 : 0); }
  __host__ __device__ static constexpr int nsbits(int s) { return s == 0 ? 0 : nsbits(s - 1) + bits(s - 1); }
  // offset of stage s in the twiddle table (stage 0 has none)
  __host__ __device__ static constexpr int off(int s) {
    return s <= 1 ? 0 : off(s - 1) + ((1 << bits(s - 1)) - 1) * (1 << nsbits(s - 1));
  }
  __host__ __device__ static constexpr int entries() { return off(S); }
};

// One Stockham stage over NSEQ sequences.  Acc maps (sequence, position) to a
// shared-memory slot; tw is this stage's part of the twiddle table.
template <int N, int E, int R, int NS, bool LAST, int SIGN, int NSEQ, class T, class Acc>
__device__ __forceinline__ void fft_stage(cx<T> (&v)[NSEQ][E], int t,
                                          const typename TwType<T>::type *__restrict__ tw, const Acc &acc) {
  constexpr int TT = N / E;
  constexpr int B = E / R;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int jv = t + b * TT;
    const int k = jv & (NS - 1);
#pragma unroll
    for (int q = 0; q < NSEQ; ++q) {
      cx<T> u[R];
#pragma unroll
      for (int r = 0; r < R; ++r) u[r] = v[q][b + r * B];
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = twiddle<SIGN, T>(u[r], tw[(r - 1) * NS + k]);
      }
      dft<R, SIGN>(u);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][b + r * B] = u[r];
      } else {
        const int base = (jv / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) acc.st(q, base + r * NS, u[r]);
      }
    }
  }
}

template <int LOGN, int LOGE, int SIGN, int NSEQ, int STAGE, class T, class Acc>
__device__ __forceinline__ void fft_stages(cx<T> (&v)[NSEQ][1 << LOGE], int t,
                                           const typename TwType<T>::type *__restrict__ tw, const Acc &acc) {
  using P = Plan<LOGN, LOGE>;
  if constexpr (STAGE < P::S) {
    constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
    constexpr int R = 1 << P::bits(STAGE);
    constexpr int NS = 1 << P::nsbits(STAGE);
    constexpr bool LAST = (STAGE == P::S - 1);
    fft_stage<N, E, R, NS, LAST, SIGN, NSEQ>(v, t, tw + P::off(STAGE), acc);
    if constexpr (!LAST) {
      acc.sync();
#pragma unroll
      for (int q = 0; q < NSEQ; ++q)
#pragma unroll
        for (int m = 0; m < E; ++m) v[q][m] = acc.ld(q, t + m * TT);
      acc.sync();
      fft_stages<LOGN, LOGE, SIGN, NSEQ, STAGE + 1>(v, t, tw, acc);
    }
  }
}

// Length-2^LOGN transform of NSEQ sequences held as described above; tw_table
// is the plan's twiddle table (Plan<LOGN, LOGE>::entries() entries).
// SIGN = -1 forward (unnormalised), +1 inverse (unnormalised).  Must be called
// by every thread that acc.sync() synchronises (the block, or the warp when
// all exchange partners of a sequence share a warp).
template <int LOGN, int LOGE, int SIGN, int NSEQ, class T, class Acc>
__device__ __forceinline__ void block_fft(cx<T> (&v)[NSEQ][1 << LOGE], int t, const void *tw_table,
                                          const Acc &acc) {
  const typename TwType<T>::type *tw = reinterpret_cast<const typename TwType<T>::type *>(tw_table);
  fft_stages<LOGN, LOGE, SIGN, NSEQ, 0>(v, t, tw, acc);
}

}  // namespace spgpe
