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
// Radix plan: S = ceil(LOGN / LOGE) stages, log2 radices split as evenly as
// possible (2048 = 16*16*8 at E = 16, 256 = 16*16, 64 = 8*8, ...).
#pragma once
#include <cuda_runtime.h>

namespace spgpe {

template <class T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <class T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.re * s, a.im * s}; }
template <class T> __device__ __forceinline__ T cabs2(cx<T> a) { return a.re * a.re + a.im * a.im; }

// a * exp(SIGN * 2 pi i M / 16) for a compile-time M in [0, 8).  The cosines
// and sines of multiples of pi/8 are written out to 20 digits and rounded
// once to T.
template <int SIGN, int M, class T>
__device__ __forceinline__ cx<T> w16(cx<T> a) {
  constexpr double C1 = 0.92387953251128675613;  // cos(pi/8)
  constexpr double S1 = 0.38268343236508977173;  // sin(pi/8)
  constexpr double H = 0.70710678118654752440;   // cos(pi/4)
  const T c1 = T(C1), s1 = T(S1), h = T(H);
  const T sg = T(SIGN);
  if constexpr (M == 0) {
    return a;
  } else if constexpr (M == 4) {
    return {-sg * a.im, sg * a.re};
  } else if constexpr (M == 2) {
    return {(a.re - sg * a.im) * h, (a.im + sg * a.re) * h};
  } else if constexpr (M == 6) {
    return {(-a.re - sg * a.im) * h, (-a.im + sg * a.re) * h};
  } else {
    // cos/sin of M*pi/8 for M = 1, 3, 5, 7
    const T c = (M == 1) ? c1 : (M == 3) ? s1 : (M == 5) ? -s1 : -c1;
    const T s = sg * ((M == 1 || M == 7) ? s1 : c1);
    return {a.re * c - a.im * s, a.re * s + a.im * c};
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
  static constexpr int S = (LOGN + LOGE - 1) / LOGE;
  __host__ __device__ static constexpr int bits(int s) { return LOGN / S + (s < LOGN % S ? 1 : 0); }
  __host__ __device__ static constexpr int nsbits(int s) { return s == 0 ? 0 : nsbits(s - 1) + bits(s - 1); }
};

// One Stockham stage over NSEQ sequences.  Acc maps (sequence, position) to a
// shared-memory slot; tw[m] = exp(-2 pi i m / N) is the forward root table.
template <int N, int E, int R, int NS, bool LAST, int SIGN, int NSEQ, class T, class Acc>
__device__ __forceinline__ void fft_stage(cx<T> (&v)[NSEQ][E], int t, const cx<T> *__restrict__ tw,
                                          const Acc &acc) {
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
        for (int r = 1; r < R; ++r) {
          cx<T> w = tw[(r * k) * (N / (NS * R))];
          if (SIGN > 0) w.im = -w.im;
          u[r] = cmul(u[r], w);
        }
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
__device__ __forceinline__ void fft_stages(cx<T> (&v)[NSEQ][1 << LOGE], int t, const cx<T> *__restrict__ tw,
                                           const Acc &acc) {
  using P = Plan<LOGN, LOGE>;
  if constexpr (STAGE < P::S) {
    constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
    constexpr int R = 1 << P::bits(STAGE);
    constexpr int NS = 1 << P::nsbits(STAGE);
    constexpr bool LAST = (STAGE == P::S - 1);
    fft_stage<N, E, R, NS, LAST, SIGN, NSEQ>(v, t, tw, acc);
    if constexpr (!LAST) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < NSEQ; ++q)
#pragma unroll
        for (int m = 0; m < E; ++m) v[q][m] = acc.ld(q, t + m * TT);
      __syncthreads();
      fft_stages<LOGN, LOGE, SIGN, NSEQ, STAGE + 1>(v, t, tw, acc);
    }
  }
}

// Length-2^LOGN transform of NSEQ sequences held as described above.
// SIGN = -1 forward (unnormalised), +1 inverse (unnormalised).  Must be called
// by every thread of the block (it synchronises the block between stages).
template <int LOGN, int LOGE, int SIGN, int NSEQ, class T, class Acc>
__device__ __forceinline__ void block_fft(cx<T> (&v)[NSEQ][1 << LOGE], int t, const cx<T> *__restrict__ tw,
                                          const Acc &acc) {
  fft_stages<LOGN, LOGE, SIGN, NSEQ, 0>(v, t, tw, acc);
}

}  // namespace spgpe
