// Fused TSSP passes for the two-component GPE (templates; instantiated per
// precision in kernels_row.cu / kernels_col.cu).
//
// One step S(dt) = R(dt/2) F^-1 K(dt) F R(dt/2) (Sec. 3.2, Eq. 13) is run as
//   row pass    : [inverse x-FFT] -> R(dt/2) [-> R(dt/2) of the next step] -> x-FFT
//   column pass : y-FFT -> K(dt) -> inverse y-FFT
// so psi crosses HBM twice per real-time step.  The row pass holds both
// components of a row in registers (R mixes them through X = exp(-i tau
// Omega sigma_x / 2) and the g12 density); the column pass holds one
// component of C adjacent columns (K is diagonal in spin).  Imaginary time
// splits the row pass at the renormalisation point: pass A ends the step and
// produces FP64 atom-number partials, the last block of each instance turns
// them into the scale, and pass B applies it before the next R(dt/2).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "async_copy.cuh"
#include "fastmath.cuh"
#include "fft_core.cuh"
#include "internal.h"

namespace spgpe {

template <class T>
struct alignas(4 * sizeof(T)) q4 {
  T x, y, z, w;
};

// ------------------------------------------------------------ math helpers

// No factor of the step may change |psi| by a fixed, rounding-made amount
// each time it is applied: such errors are systematic for slowly varying
// phases and add up over thousands of steps.  So the kinetic factor K is
// applied as z + (f - 1) z with f - 1 evaluated to full relative precision
// (f - 1 = -2 sin^2(h) + 2i sin(h) cos(h), h the half phase; expm1 in
// imaginary time), the small part first and z added last; the real-time D
// phase and the Raman rotation X (in imaginary time the hyperbolic rotation)
// are three-shear rotations, whose determinant is one whatever the rounding
// of their constants.  The operations are written with explicit fma so that
// every kernel that applies them rounds identically.

// Shear constants (tanh(a/2), sinh a) of the hyperbolic rotation by a (the
// imaginary-time X of a 2D Omega entry), from expm1 to full relative
// precision: tanh(a/2) = e / (e + 2) and sinh a = (e - expm1(-a)) / 2 with
// e = expm1(a).
template <class T> __device__ __forceinline__ void hrot_consts(T a, T &t, T &s) {
  if constexpr (sizeof(T) == 4) {
    const T e = expm1_f(a), f = expm1_f(-a);
    t = e / (e + T(2));
    s = T(0.5) * (e - f);
  } else {
    t = tanh(T(0.5) * a);
    s = sinh(a);
  }
}

// Imaginary-time X(theta) = exp(-theta sigma_x): the hyperbolic rotation
// [[cosh, -sinh], [-sinh, cosh]] of the planes (Re u, Re d) and (Im u, Im d),
// each as three shears x -= t y; y -= s x; x -= t y with t = tanh(theta/2),
// s = sinh(theta) (their product is [[1 + t s, -t (2 + t s)], [-s, 1 + t s]]
// and 1 + t s = cosh theta); 6 fma, determinant one.
template <class T> __device__ __forceinline__ void opXh(cx<T> &u, cx<T> &d, T t, T s) {
  const T x1 = d_fma(-t, d.re, u.re);
  const T y1 = d_fma(-s, x1, d.re);
  const T x2 = d_fma(-t, y1, x1);
  const T p1 = d_fma(-t, d.im, u.im);
  const T q1 = d_fma(-s, p1, d.im);
  const T p2 = d_fma(-t, q1, p1);
  u = {x2, p2};
  d = {y1, q1};
}

// z <- z + z w for a complex w = f - 1 (small part first, z added last).
template <class T> __device__ __forceinline__ cx<T> add_mul1(cx<T> z, cx<T> w) {
  return {z.re + d_fma(z.re, w.re, -(z.im * w.im)), z.im + d_fma(z.re, w.im, z.im * w.re)};
}

// expm1 of the single-precision general tier, out of line (imaginary-time
// warps whose interaction exponent exceeds the series bound: rare, so one
// shared copy keeps the passes within the instruction cache).
static __device__ __noinline__ float expm1_general(float x) { return expm1_f(x); }
__device__ __forceinline__ double expm1_general(double x) { return expm1(x); }

// D(tau): diagonal potential + mean-field phase (decay), densities on entry.
// htau = -tau/2 in real time (the half phase), -tau in imaginary time; the
// couplings arrive multiplied by it (gh11 = htau g11, ...: per instance, formed
// once by the caller).
// Real time: vu, vd are htau (V +- delta/2), so that the half phase is
// h = vu + gh11 rho_up + gh12 rho_dn (resp. down), the whole exponent.
// Imaginary time: vu, vd are the potential factors exp(-tau (V +- delta/2))
// (from the step tables) and only the interaction exponent -tau (g11 rho_up +
// g12 rho_dn) (resp. down) goes through expm1: exp(-tau (V + g rho)) =
// exp(-tau V) (1 + expm1(-tau g rho)).
// TIER (the caller has checked it for every point of the warp): real time
// 0: |h| < 1/64, 1: |h| < 1/8; imaginary time (h the interaction exponent)
// 0: |h| < 1/4, 1: |h| < 1/2; so the series need no range reduction; 2: any
// phase.  FP64 always takes the library functions.
template <bool IMAG, int TIER = 2, class T>
__device__ __forceinline__ void opD(cx<T> &u, cx<T> &d, T vu, T vd, T gh11, T gh22, T gh12) {
  constexpr bool F32 = sizeof(T) == 4;
  const T ru = d_fma(u.re, u.re, u.im * u.im), rd = d_fma(d.re, d.re, d.im * d.im);
  if constexpr (IMAG) {
    const T hu = d_fma(gh12, rd, gh11 * ru), hd = d_fma(gh12, ru, gh22 * rd);
    T fu, fd;
    if constexpr (F32 && TIER == 0) {
      fu = expm1_quarter(hu);
      fd = expm1_quarter(hd);
    } else if constexpr (F32 && TIER == 1) {
      fu = expm1_small(hu);
      fd = expm1_small(hd);
    } else {
      fu = expm1_general(hu);
      fd = expm1_general(hd);
    }
    const T au = d_fma(vu, fu, vu), ad = d_fma(vd, fd, vd);  // exp(-tau V) (1 + expm1(-tau g rho))
    u = {u.re * au, u.im * au};
    d = {d.re * ad, d.im * ad};
  } else {
    const T hu = d_fma(gh12, rd, d_fma(gh11, ru, vu));
    const T hd = d_fma(gh12, ru, d_fma(gh22, rd, vd));
    // the phases exp(-i tau e) as three-shear rotations by 2 h
    // (determinant one: no systematic change of |psi| from rounded constants)
    T tu, su, td, sd;
    if constexpr (F32 && TIER == 0) {
      shear_consts_2h_tiny(hu, tu, su);
      shear_consts_2h_tiny(hd, td, sd);
    } else if constexpr (F32 && TIER == 1) {
      shear_consts_2h_small(hu, tu, su);
      shear_consts_2h_small(hd, td, sd);
    } else {
      bool nu, nd;
      shear_consts_2h(hu, tu, su, nu);
      shear_consts_2h(hd, td, sd, nd);
      // a rotation by 2r + pi: negate (commutes with the rotation by 2r)
      if (nu) u = {-u.re, -u.im};
      if (nd) d = {-d.re, -d.im};
    }
    u = shear_rot(u, tu, su);
    d = shear_rot(d, td, sd);
  }
}

// Real-time X(theta) = exp(-i theta sigma_x) as two independent plane
// rotations: (Re u, Im d) by -theta and (Im u, Re d) by +theta, each with
// three shears (t = tan(theta/2), s = sin(theta)); 6 fma, determinant one.
template <class T> __device__ __forceinline__ void opXr(cx<T> &u, cx<T> &d, T t, T s) {
  const T x1 = d_fma(t, d.im, u.re);
  const T y1 = d_fma(-s, x1, d.im);
  const T x2 = d_fma(t, y1, x1);
  const T p1 = d_fma(-t, d.re, u.im);
  const T q1 = d_fma(s, p1, d.re);
  const T p2 = d_fma(-t, q1, p1);
  u = {x2, p2};
  d = {q1, y1};
}

// X constants at one point: the separate rotations of the y piece, the x
// piece and the 2D piece of the angle (rotations about sigma_x commute), each
// applied only when that piece is present; (tan, sin) of the half and whole
// angle in real time, (tanh, sinh) in imaginary time.
template <class T> struct XPoint {
  T m, s;          // y piece
  T tx, sx;        // x piece
  T t2, s2;        // 2D piece
  bool n2;         // real time: the 2D piece rotates by 2r + pi, negate afterwards
};

template <bool IMAG, class T>
__device__ __forceinline__ void applyX(cx<T> &u, cx<T> &d, const XPoint<T> &x, int pieces) {
  auto rot = [&](T t, T s) {
    if constexpr (IMAG) opXh(u, d, t, s); else opXr(u, d, t, s);
  };
  if (pieces & 1) rot(x.m, x.s);
  if (pieces & 2) rot(x.tx, x.sx);
  if (pieces & 4) {
    rot(x.t2, x.s2);
    if (!IMAG && x.n2) {
      u = {-u.re, -u.im};
      d = {-d.re, -d.im};
    }
  }
}

// Real-time X applied twice in a row (the closing R(dt/2) of one step meets
// the opening R(dt/2) of the next): the y piece as one rotation by the doubled
// angle when (tm, sm) are its shear constants (ymerge), the other pieces
// twice (their negations cancel).
template <class T>
__device__ __forceinline__ void applyX2(cx<T> &u, cx<T> &d, const XPoint<T> &x, int pieces, bool ymerge, T tm,
                                        T sm) {
  if (pieces & 1) {
    if (ymerge) {
      opXr(u, d, tm, sm);
    } else {
      opXr(u, d, x.m, x.s);
      opXr(u, d, x.m, x.s);
    }
  }
  if (pieces & 2) {
    opXr(u, d, x.tx, x.sx);
    opXr(u, d, x.tx, x.sx);
  }
  if (pieces & 4) {
    opXr(u, d, x.t2, x.s2);
    opXr(u, d, x.t2, x.s2);
  }
}

// Shear constants of the doubled angle from (t, s) = (tan(a/2), sin a):
// cos a = 1 - t s, so tan a = s / (1 - t s) and sin 2a = 2 s (1 - t s).
// Valid (ymerge) while |a| < pi/4, i.e. cos a > 1/sqrt 2.
template <class T> __device__ __forceinline__ bool x_double(T t, T s, T &tm, T &sm) {
  const T c = d_fma(-t, s, T(1));
  tm = s / c;
  sm = T(2) * s * c;
  return c > T(0.70710678118654752);
}

// X constants at point (x, y): px, ty are the x and y step-table entries,
// q2z the 2D Omega (or 0), xang = dt/8.
template <bool IMAG, class T>
__device__ __forceinline__ XPoint<T> xpoint(const q4<T> &px, const q4<T> &ty, bool has2d, T q2z, T xang) {
  XPoint<T> r;
  r.m = ty.z;
  r.s = ty.w;
  r.tx = px.z;
  r.sx = px.w;
  r.t2 = r.s2 = T(0);
  r.n2 = false;
  if (has2d) {
    if constexpr (IMAG) hrot_consts(q2z * xang, r.t2, r.s2);
    else shear_consts_2h(T(0.5) * q2z * xang, r.t2, r.s2, r.n2);
  }
  return r;
}

// --------------------------------------------------------- block reductions

// Deterministic block sum of K doubles (fixed shuffle tree, fixed warp order).
// Every thread must call it; the result is valid in thread 0.
template <int K> __device__ __forceinline__ void block_sum(double (&v)[K]) {
  __shared__ double red[K][32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[k][w] = v[k];
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = (l < nw) ? red[k][l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  __syncthreads();
}

// ---------------------------------------------------- shared-memory layouts

// WARP_LOCAL: every thread that exchanges values with this one through
// shared memory is in its warp (a row's threads never straddle warps), so the
// stages synchronise with a warp barrier over `mask` instead of the block.
template <class T, bool WARP_LOCAL = false> struct RowAcc {
  static constexpr int SH = pad_shift(sizeof(cx<T>));
  cx<T> *base;
  int stride;
  unsigned mask;
  __device__ __forceinline__ void st(int q, int p, cx<T> v) const { base[q * stride + p + (p >> SH)] = v; }
  __device__ __forceinline__ cx<T> ld(int q, int p) const { return base[q * stride + p + (p >> SH)]; }
  __device__ __forceinline__ void sync() const {
    if constexpr (WARP_LOCAL) __syncwarp(mask); else __syncthreads();
  }
};

template <class T> struct ColAcc {
  static constexpr int SH = pad_shift(sizeof(cx<T>));
  cx<T> *base;
  int C, c;
  __device__ __forceinline__ int idx(int p) const { const int e = p * C + c; return e + (e >> SH); }
  __device__ __forceinline__ void st(int, int p, cx<T> v) const { base[idx(p)] = v; }
  __device__ __forceinline__ cx<T> ld(int, int p) const { return base[idx(p)]; }
  __device__ __forceinline__ static void sync() { __syncthreads(); }
};

// Same layout with the tile width known at compile time: for C a multiple of
// the 128-byte line (in elements) the padding term is linear in p and every
// exchange address folds into a per-thread base plus an immediate offset.
template <class T, int C> struct ColAccC {
  static constexpr int SH = pad_shift(sizeof(cx<T>));
  cx<T> *base;  // already offset by the thread's column
  __device__ __forceinline__ static int idx(int p) { return p * C + ((p * C) >> SH); }
  __device__ __forceinline__ void st(int, int p, cx<T> v) const { base[idx(p)] = v; }
  __device__ __forceinline__ cx<T> ld(int, int p) const { return base[idx(p)]; }
  __device__ __forceinline__ static void sync() { __syncthreads(); }
};

// ------------------------------------------------------------- row pass
//
// Each row is held by 2*TT threads: TT threads per component, E values each.
// Within a warp the two components sit in lane groups `half` apart (lanes
// 0..half-1 component up, the next half lanes component down, repeated), so
// the partner holding the other component of the same positions is lane ^ half.
// The transforms run on one component per thread.  For the pointwise R
// operator, which needs both components of a point, partners swap half of
// their values with shuffles: the up-thread then owns positions m < E/2 of
// both components, the down-thread positions m >= E/2; they swap back after.

// R_end and/or R_start at one point x of row y (both components).
// MERGE (the fused real-time pass): X D X X D X with the middle X X as one
// doubled X (exact: the two factors are the same rotation about sigma_x).
// TIER: the phase tier of opD, one instantiation per tier so that each warp
// runs straight-line code.  SIMPLE: the common layout, fixed at compile time
// so that no point tests it: no 2D potential table, the Raman rotation in the
// y piece only (an absent rotation is the exact identity), and in real time
// the doubled y rotation valid (ymerge).  gh11, gh22, gh12 are the couplings
// times htau; the real-time step tables hold htau (V +- delta/2).
template <class T, int N, int F, int TIER, bool SIMPLE>
__device__ __forceinline__ void r_one(cx<T> &u, cx<T> &d, int x, int y, const q4<T> *tab, const q4<T> &ty,
                                      const q4<T> *p2, T gh11, T gh22, T gh12, T htau, T xang, int pieces,
                                      bool ymerge, T tm, T sm, T su, T sd, T (&nsum)[2]) {
  constexpr bool IMAG = (F & F_IMAG) != 0;
  constexpr bool MERGE = !IMAG && (F & F_REND) && (F & F_RSTART) && !(F & F_PART);
  if constexpr (SIMPLE) {
    p2 = nullptr;
    pieces = 1;
    ymerge = true;
  }
  const q4<T> px = tab[x];
  T vu, vd, q2z = T(0);
  if constexpr (IMAG) {  // potential factors exp(-tau (V +- delta/2)) of the separable pieces
    vu = px.x * ty.x;
    vd = px.y * ty.y;
  } else {
    vu = px.x + ty.x;
    vd = px.y + ty.y;
  }
  if (p2) {
    const q4<T> q = p2[(long)y * N + x];
    if constexpr (IMAG) {
      vu *= exp(htau * q.x);
      vd *= exp(htau * q.y);
    } else {
      vu = d_fma(htau, q.x, vu);
      vd = d_fma(htau, q.y, vd);
    }
    q2z = q.z;
  }
  const XPoint<T> xc = xpoint<IMAG, T>(px, ty, p2 != nullptr, q2z, xang);
  if constexpr (MERGE) {
    applyX<false>(u, d, xc, pieces);
    opD<false, TIER>(u, d, vu, vd, gh11, gh22, gh12);
    applyX2(u, d, xc, pieces, ymerge, tm, sm);
    opD<false, TIER>(u, d, vu, vd, gh11, gh22, gh12);
    applyX<false>(u, d, xc, pieces);
  } else {
    if constexpr (F & F_REND) {
      applyX<IMAG>(u, d, xc, pieces);
      opD<IMAG, TIER>(u, d, vu, vd, gh11, gh22, gh12);
      applyX<IMAG>(u, d, xc, pieces);
    }
    if constexpr (F & F_PART) {
      nsum[0] += cabs2(u);
      nsum[1] += cabs2(d);
    }
    if constexpr (F & F_LAG) {
      u = cscale(u, su);
      d = cscale(d, sd);
    }
    if constexpr (F & F_RSTART) {
      applyX<IMAG>(u, d, xc, pieces);
      opD<IMAG, TIER>(u, d, vu, vd, gh11, gh22, gh12);
      applyX<IMAG>(u, d, xc, pieces);
    }
  }
}

// R_end and/or R_start at this thread's K points (both components): pu[j],
// pd[j] at x = t + (j + jo) * TT of row y; as r_one.
template <class T, int LOGN, int LOGE, int F, int TIER, bool SIMPLE, int K>
__device__ __forceinline__ void r_points(cx<T> (&pu)[K], cx<T> (&pd)[K], int t, int jo, int y, const q4<T> *tab,
                                         const q4<T> &ty, const q4<T> *p2, T gh11, T gh22, T gh12, T htau, T xang,
                                         int pieces, bool ymerge, T tm, T sm, T su, T sd, T (&nsum)[2]) {
  constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
#pragma unroll
  for (int j = 0; j < K; ++j)
    r_one<T, N, F, TIER, SIMPLE>(pu[j], pd[j], t + (j + jo) * TT, y, tab, ty, p2, gh11, gh22, gh12, htau, xang,
                                 pieces, ymerge, tm, sm, su, sd, nsum);
}

// The pointwise part of the row pass, R_end and/or R_start, on K points per
// thread with both components in registers (pu[j], pd[j] at x = t + (j + jo)
// * TT of row y).  The lanes in mask hold together the points whose phase
// bound picks one series tier for all of them (the same point sets in every
// variant of the pass, so that they round alike).  Adds the thread's
// atom-number partials of the R_end result to nsum when F has F_PART.
template <class T, int LOGN, int LOGE, int F, int K>
__device__ __forceinline__ void r_apply(cx<T> (&pu)[K], cx<T> (&pd)[K], int t, int jo, unsigned mask, int inst, int y,
                                        const q4<T> *tab, const RowArgs &a, T (&nsum)[2]) {
  constexpr bool IMAG = (F & F_IMAG) != 0;
  // (bounds-checked build: a bad row index is recorded and replaced by 0, so
  // that every thread still reaches the warp's barriers)
  const long tyi = in_bounds(a.flags, (long)inst * a.ny + y, (long)a.ninst * a.ny) ? (long)inst * a.ny + y : 0;
  const q4<T> ty = reinterpret_cast<const q4<T> *>(a.taby)[tyi];
  const q4<T> *p2 = reinterpret_cast<const q4<T> *>(a.pot2d);
  const T *gp = reinterpret_cast<const T *>(a.gparT) + 4 * inst;
  const T g11 = gp[0], g22 = gp[1], g12 = gp[2];
  T htau, xang;
  if constexpr (sizeof(T) == 4) { htau = a.htau_f; xang = a.xang_f; } else { htau = a.htau_d; xang = a.xang; }
  const T gh11 = htau * g11, gh22 = htau * g22, gh12 = htau * g12;
  const int pieces = (a.omega_pieces & 3) | (p2 ? 4 : 0);
  const T gmax = fmax(fabs(g11), fabs(g22)) + fabs(g12);
  T tm = T(0), sm = T(0);
  T su = T(1), sd = T(1);
  if constexpr ((F & F_LAG) != 0) {
    su = reinterpret_cast<const T *>(a.scale_pred_t)[2 * inst];
    sd = reinterpret_cast<const T *>(a.scale_pred_t)[2 * inst + 1];
  }
  bool ymerge = false;
  if constexpr (!IMAG && (F & F_REND) && (F & F_RSTART)) ymerge = x_double(ty.z, ty.w, tm, sm);
  // One phase tier per lane group: the shortest series whose range holds
  // |htau e| at every point of the group.  e <= Vb + G rho_tot with Vb = max
  // |V +- delta/2| of the instance and G = max(|g11|, |g22|) + |g12|;
  // rho_tot = |u|^2 + |d|^2 at a point is left unchanged by real-time R (5 %
  // margin for the imaginary-time X).
  T rmax = T(0);
#pragma unroll
  for (int j = 0; j < K; ++j) rmax = fmax(rmax, d_fma(pu[j].re, pu[j].re, pu[j].im * pu[j].im) +
                                                    d_fma(pd[j].re, pd[j].re, pd[j].im * pd[j].im));
  // (the lagged pass scales the densities between R_end and R_start by the
  // squared predicted scale)
  if constexpr ((F & F_LAG) != 0) rmax *= fmax(T(1), fmax(su * su, sd * sd));
  // (imaginary time: the potential factors come from tables, so only the
  // interaction exponent is bounded; real time: the whole phase)
  const T hb = fabs(htau) * ((IMAG ? T(0) : gp[3]) + gmax * T(1.05) * rmax);
  const bool small = __all_sync(mask, hb < (IMAG ? T(0.5) : T(0.125)));
  const bool tiny = __all_sync(mask, hb < (IMAG ? T(0.25) : T(0.015625)));
  // the common layout (r_one's SIMPLE), decided for the whole group
  constexpr bool YM = !IMAG && (F & F_REND) && (F & F_RSTART);
  const bool simple = __all_sync(mask, p2 == nullptr && (a.omega_pieces & 2) == 0 && (!YM || ymerge));
#define SPGPE_R_POINTS(TIER, S)                                                                                      \
  r_points<T, LOGN, LOGE, F, TIER, S, K>(pu, pd, t, jo, y, tab, ty, p2, gh11, gh22, gh12, htau, xang, pieces, ymerge, \
                                         tm, sm, su, sd, nsum)
  if constexpr (sizeof(T) == 8) {
    if (simple)
      SPGPE_R_POINTS(2, true);
    else
      SPGPE_R_POINTS(2, false);
  } else if (simple) {
    if (tiny)
      SPGPE_R_POINTS(0, true);
    else if (small)
      SPGPE_R_POINTS(1, true);
    else
      SPGPE_R_POINTS(2, true);
  } else {
    if (tiny)
      SPGPE_R_POINTS(0, false);
    else if (small)
      SPGPE_R_POINTS(1, false);
    else
      SPGPE_R_POINTS(2, false);
  }
#undef SPGPE_R_POINTS
}

// Row-pass compute on registers already loaded: v holds this thread's
// component at positions t + m*TT of row y.  tab points at the instance's
// x step table (global or shared memory).  Adds this thread's atom-number
// partials of the R_end result (its H points of both components, summed in
// the working precision) to nsum when F has F_PART.
template <class T, int LOGN, int LOGE, int F, class Acc>
__device__ __forceinline__ void row_compute(cx<T> (&v)[1][1 << LOGE], int t, int comp, unsigned mask, int half,
                                            int inst, int y, const Acc &acc, const q4<T> *tab,
                                            const RowArgs &a, T (&nsum)[2]) {
  constexpr int E = 1 << LOGE, H = E / 2;
  if constexpr (F & F_IFFT) block_fft<LOGN, LOGE, +1, 1>(v, t, a.tw, acc);
  if constexpr (F & F_SCALE) {
    const T sc = reinterpret_cast<const T *>(a.scale_t)[2 * inst + comp];
#pragma unroll
    for (int m = 0; m < E; ++m) v[0][m] = cscale(v[0][m], sc);
  }
  if constexpr (F & (F_REND | F_RSTART)) {
    // gather: (pu[j], pd[j]) = both components at position m = j + comp*H
    cx<T> pu[H], pd[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const cx<T> snd = comp ? v[0][j] : v[0][H + j];
      const cx<T> rcv = {__shfl_xor_sync(mask, snd.re, half), __shfl_xor_sync(mask, snd.im, half)};
      pu[j] = comp ? rcv : v[0][j];
      pd[j] = comp ? v[0][H + j] : rcv;
    }
    r_apply<T, LOGN, LOGE, F, H>(pu, pd, t, comp * H, mask, inst, y, tab, a, nsum);
    // scatter back to one component per thread
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const cx<T> snd = comp ? pu[j] : pd[j];
      const cx<T> rcv = {__shfl_xor_sync(mask, snd.re, half), __shfl_xor_sync(mask, snd.im, half)};
      v[0][j] = comp ? rcv : pu[j];
      v[0][H + j] = comp ? pd[j] : rcv;
    }
  }
  if constexpr (F & F_FFT) block_fft<LOGN, LOGE, -1, 1>(v, t, a.tw, acc);
}

// Sum of a per-thread pair over the block into thread 0: in single
// precision each warp first adds its lanes' values in a fixed FP32 tree (the
// summands are non-negative, so the relative error stays below 13 units of
// FP32 rounding for 8 points per lane), and the warps' totals go on in FP64;
// double precision sums in FP64 throughout (block_sum).
template <class T> __device__ __forceinline__ void block_sum_pair(const T (&v)[2], double (&out)[2]) {
  if constexpr (sizeof(T) == 4) {
    __shared__ double red2[2][32];
    float w0 = v[0], w1 = v[1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      w0 += __shfl_xor_sync(0xffffffffu, w0, o);
      w1 += __shfl_xor_sync(0xffffffffu, w1, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
      red2[0][w] = double(w0);
      red2[1][w] = double(w1);
    }
    __syncthreads();
    out[0] = out[1] = 0.0;
    if (threadIdx.x == 0) {
      const int nw = (blockDim.x + 31) >> 5;
      for (int k = 0; k < nw; ++k) {
        out[0] += red2[0][k];
        out[1] += red2[1][k];
      }
    }
    __syncthreads();
  } else {
    out[0] = v[0];
    out[1] = v[1];
    block_sum<2>(out);
  }
}

// Count a finished row group: an atomic add with release-acquire ordering at
// GPU scope, so the group's partial sums written before it are visible to the
// group that sees the final count (and that group sees every other group's).
__device__ __forceinline__ unsigned count_group(unsigned *counter) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(counter) : "memory");
  return old;
}

// The last row group of an instance publishes its renormalisation scale: in
// FP64, in the working precision (what F_SCALE and F_LAG multiply by), and
// for a lagged pass the column pass's correction scale / predicted scale; it
// then rearms the instance's counter.
template <class T> __device__ __forceinline__ void write_scale(const RowArgs &a, int inst, double s0, double s1) {
  a.scale[2 * inst] = s0;
  a.scale[2 * inst + 1] = s1;
  T *st = reinterpret_cast<T *>(a.scale_t);
  st[2 * inst] = T(s0);
  st[2 * inst + 1] = T(s1);
  if (a.cfac) {
    T *cf = reinterpret_cast<T *>(a.cfac);
    cf[2 * inst] = T(s0 / a.scale_pred[2 * inst]);
    cf[2 * inst + 1] = T(s1 / a.scale_pred[2 * inst + 1]);
  }
  a.counters[inst] = 0u;
}

// Atom-number partials of one row group; the last group of the instance to
// finish reduces them in a fixed order (FP64) and writes the
// renormalisation scale (Sec. 3.2).  Called by every thread of the block.
template <class T>
__device__ __forceinline__ void row_partials(const RowArgs &a, int inst, int group, int ngroups, const T (&tsum)[2]) {
  __shared__ int s_last;
  double nsum[2];
  block_sum_pair<T>(tsum, nsum);
  if (threadIdx.x == 0) {
    if (in_bounds(a.flags, ((long)inst * ngroups + group) * 2 + 1, (long)a.ninst * a.ny * 2) &&
        in_bounds(a.flags, inst, a.ninst)) {
      a.partials[((long)inst * ngroups + group) * 2] = nsum[0];
      a.partials[((long)inst * ngroups + group) * 2 + 1] = nsum[1];
    }
    const unsigned prev = count_group(&a.counters[inst]);
    s_last = (prev == (unsigned)ngroups - 1u);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    double tot[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < ngroups; b += blockDim.x) {
      tot[0] += __ldcg(&a.partials[((long)inst * ngroups + b) * 2]);
      tot[1] += __ldcg(&a.partials[((long)inst * ngroups + b) * 2 + 1]);
    }
    block_sum<2>(tot);
    if (threadIdx.x == 0) {
      const double nu = tot[0] * a.wgt, nd = tot[1] * a.wgt;
      double s0, s1;
      if (a.norm_mode == 1) {
        s0 = sqrt(a.tgt0 / nu);
        s1 = sqrt(a.tgt1 / nd);
      } else {
        s0 = s1 = sqrt((a.tgt0 + a.tgt1) / (nu + nd));
      }
      if (!isfinite(s0) || !isfinite(s1)) atomicOr(a.flags, 1);
      write_scale<T>(a, inst, s0, s1);
    }
  }
  __syncthreads();
}

// Thread placement of the row pass (see above).  With TT <= 16 threads per
// component a row lies in one warp (or in the whole block, below 32 threads).
__host__ __device__ constexpr bool row_warp_local(int tt) { return tt <= 16; }
struct RowPlace {
  int half, comp, lrow, t;
  unsigned mask;
};
template <int TT> __device__ __forceinline__ RowPlace row_place() {
  RowPlace r;
  r.half = min(16, (int)blockDim.x / 2);
  r.mask = blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u);
  const int tx = threadIdx.x;
  r.comp = (tx / r.half) & 1;
  const int tp = (tx % r.half) + r.half * (tx / (2 * r.half));
  r.lrow = tp / TT;
  r.t = tp - r.lrow * TT;
  return r;
}

// Largest block of the plain row pass: kRowMaxThreads, or the 2*TT threads of
// one row when that is more (4096-point rows; 2048-point complex128 rows).
__host__ __device__ constexpr int row_block_max(int logn, int loge) {
  return 2 * ((1 << logn) >> loge) > kRowMaxThreads ? 2 * ((1 << logn) >> loge) : kRowMaxThreads;
}

template <class T, int LOGN, int LOGE, int F>
__global__ void __launch_bounds__(row_block_max(LOGN, LOGE), sizeof(T) == 4 && LOGN <= 11 ? 3 : 1)
row_pass(const RowArgs a) {
  constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
  const RowPlace pl = row_place<TT>();
  const int inst = blockIdx.y;
  if (a.active && !a.active[inst]) return;  // frozen instance (uniform over the block)
  const int y = blockIdx.x * a.rows + pl.lrow;
  cx<T> *p = reinterpret_cast<cx<T> *>(a.psi) + (((long)inst * 2 + pl.comp) * a.ny + y) * N;
  constexpr int PADN = row_pad_n(N, sizeof(cx<T>));
  const RowAcc<T, row_warp_local(TT)> acc{sm + pl.lrow * row_stride(N, sizeof(cx<T>)) + pl.comp * PADN, 0,
                                          pl.mask};

  const long pbase = (((long)inst * 2 + pl.comp) * a.ny + y) * N, ptotal = (long)a.ninst * 2 * a.ny * N;
  cx<T> v[1][E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[0][m] = in_bounds(a.flags, pbase + pl.t + m * TT, ptotal) ? p[pl.t + m * TT] : cx<T>{};
  T nsum[2] = {T(0), T(0)};
  row_compute<T, LOGN, LOGE, F>(v, pl.t, pl.comp, pl.mask, pl.half, inst, y, acc,
                                reinterpret_cast<const q4<T> *>(a.tabx) + (long)inst * N, a, nsum);
  if constexpr (F & F_PART) row_partials<T>(a, inst, blockIdx.x, gridDim.x, nsum);
#pragma unroll
  for (int m = 0; m < E; ++m)
    if (in_bounds(a.flags, pbase + pl.t + m * TT, ptotal)) p[pl.t + m * TT] = v[0][m];
}

// ---------------------------------------------------------- column pass

// The column pass's final factor for column group pc = 2 inst + comp: the
// inverse transform's 1/(nx ny), times the correction s_n / s_{n-1} of the
// lagged renormalisation when there is one.
template <class T> __device__ __forceinline__ T col_inv(const ColArgs &a, int pc) {
  T inv;
  if constexpr (sizeof(T) == 4) inv = a.inv_f; else inv = a.inv_d;
  return a.cfac ? inv * reinterpret_cast<const T *>(a.cfac)[pc] : inv;
}

// Column-pass compute on registers already loaded: forward y-FFT, K(dt) with
// am = a_j(kx) - 1 and bm = b(ky) - 1 (global or shared), inverse y-FFT.
// K' - 1 = (a-1)(b-1) + (a-1) + (b-1) is applied as z + (K' - 1) z and the
// exact power of two 1/(nx ny) last.
template <class T, int LOGN, int LOGE, bool IMAG, class Acc>
__device__ __forceinline__ void col_compute(cx<T> (&v)[1][1 << LOGE], int t, const Acc &acc, const void *tw,
                                            cx<T> am, const cx<T> *bm, T inv) {
  constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
  block_fft<LOGN, LOGE, -1, 1>(v, t, tw, acc);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const cx<T> b = bm[t + m * TT];
    cx<T> z = v[0][m];
    if constexpr (IMAG) {
      const T k1 = d_fma(am.re, b.re, am.re + b.re);
      z = {d_fma(z.re, k1, z.re), d_fma(z.im, k1, z.im)};
    } else {
      const cx<T> k1 = {d_fma(am.re, b.re, d_fma(-am.im, b.im, am.re + b.re)),
                        d_fma(am.re, b.im, d_fma(am.im, b.re, am.im + b.im))};
      z = add_mul1(z, k1);
    }
    if constexpr (sizeof(T) == 4) {
      const float2 zi = __fmul2_rn(make_float2(z.re, z.im), make_float2(inv, inv));
      v[0][m] = {zi.x, zi.y};
    } else {
      v[0][m] = {z.re * inv, z.im * inv};
    }
  }
  block_fft<LOGN, LOGE, +1, 1>(v, t, tw, acc);
}

template <class T, int LOGN, int LOGE, bool IMAG>
__global__ void __launch_bounds__(512) col_pass(const ColArgs a) {
  constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int C = a.C;
  const int c = threadIdx.x % C, t = threadIdx.x / C;
  const int comp = blockIdx.y, inst = blockIdx.z;
  if (a.active && !a.active[inst]) return;  // frozen instance (uniform over the block)
  const int kx = blockIdx.x * C + c;
  cx<T> *col = reinterpret_cast<cx<T> *>(a.psi) + ((long)inst * 2 + comp) * (long)N * a.nx + kx;
  const ColAcc<T> acc{reinterpret_cast<cx<T> *>(smem_raw), C, c};
  const int rs = TT * a.nx;  // element offset between a thread's rows (fits in 32 bits)

  const long cbase = ((long)inst * 2 + comp) * (long)N * a.nx + kx, ctotal = (long)a.ninst * 2 * N * a.nx;
  cx<T> v[1][E];
#pragma unroll
  for (int m = 0; m < E; ++m)
    v[0][m] = in_bounds(a.flags, cbase + t * a.nx + m * rs, ctotal) ? col[t * a.nx + m * rs] : cx<T>{};
  const long ai = ((long)inst * 2 + comp) * a.nx + kx;
  const cx<T> am = reinterpret_cast<const cx<T> *>(a.kxt)[in_bounds(a.flags, ai, (long)a.ninst * 2 * a.nx) ? ai : 0];
  const T inv = col_inv<T>(a, inst * 2 + comp);
  col_compute<T, LOGN, LOGE, IMAG>(v, t, acc, a.tw, am, reinterpret_cast<const cx<T> *>(a.kyt), inv);
#pragma unroll
  for (int m = 0; m < E; ++m)
    if (in_bounds(a.flags, cbase + t * a.nx + m * rs, ctotal)) col[t * a.nx + m * rs] = v[0][m];
}

// --------------------------------------------------------- energy passes

__device__ __forceinline__ int kbin(int i, int n) { return i < n / 2 ? i : i - n; }

// Real-space energy densities (trap, detuning, Raman, interaction, atom
// numbers) in FP64, then the forward x-FFT of both components into scratch.
template <class T, int LOGN, int LOGE>
__global__ void __launch_bounds__(2 * kRowMaxThreads) energy_row(const EnergyArgs a) {
  constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cx<T> *sm = reinterpret_cast<cx<T> *>(smem_raw);
  const int lrow = threadIdx.x / TT, t = threadIdx.x - lrow * TT;
  const int inst = blockIdx.y;
  const int y = blockIdx.x * a.rows + lrow;
  const long plane = (long)a.ny * N;
  const long off = (long)inst * 2 * plane + (long)y * N;
  const cx<T> *up = reinterpret_cast<const cx<T> *>(a.psi) + off;
  const cx<T> *dn = up + plane;
  cx<T> *oup = reinterpret_cast<cx<T> *>(a.scratch) + off;
  cx<T> *odn = oup + plane;
  const RowAcc<T> acc{sm + lrow * row_stride(N, sizeof(cx<T>)), row_pad_n(N, sizeof(cx<T>))};
  const q4<T> ry = reinterpret_cast<const q4<T> *>(a.rawy)[(long)inst * a.ny + y];
  const q4<T> *rx = reinterpret_cast<const q4<T> *>(a.rawx) + (long)inst * N;
  const q4<T> *p2 = reinterpret_cast<const q4<T> *>(a.pot2d);
  const double g11 = a.gpar[4 * inst], g22 = a.gpar[4 * inst + 1], g12 = a.gpar[4 * inst + 2];

  cx<T> v[2][E];
  double acc6[6] = {0, 0, 0, 0, 0, 0};  // trap, detuning, Raman, interaction, N_up, N_dn
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int x = t + m * TT;
    v[0][m] = up[x];
    v[1][m] = dn[x];
    const q4<T> px = rx[x];
    double V = double(px.x) + double(ry.x), de = double(px.y) + double(ry.y), Om = double(px.z) + double(ry.z);
    if (p2) {
      const q4<T> q = p2[(long)y * N + x];
      V += 0.5 * (double(q.x) + double(q.y));
      de += double(q.x) - double(q.y);
      Om += double(q.z);
    }
    const double ur = v[0][m].re, ui = v[0][m].im, dr = v[1][m].re, di = v[1][m].im;
    const double ru = ur * ur + ui * ui, rd = dr * dr + di * di;
    acc6[0] += V * (ru + rd);
    acc6[1] += 0.5 * de * (ru - rd);
    acc6[2] += Om * (ur * dr + ui * di);
    acc6[3] += 0.5 * g11 * ru * ru + 0.5 * g22 * rd * rd + g12 * ru * rd;
    acc6[4] += ru;
    acc6[5] += rd;
  }
  block_sum<6>(acc6);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) a.partials[((long)inst * gridDim.x + blockIdx.x) * 6 + k] = acc6[k];
  block_fft<LOGN, LOGE, -1, 2>(v, t, a.twx, acc);
#pragma unroll
  for (int m = 0; m < E; ++m) {
    oup[t + m * TT] = v[0][m];
    odn[t + m * TT] = v[1][m];
  }
}

// Forward y-FFT of the scratch columns and the kinetic sum
// sum_k T_j(k) |psi_hat_j(k)|^2 with T_j = k^2/2 -+ kL kx, in FP64.
template <class T, int LOGN, int LOGE>
__global__ void __launch_bounds__(512) energy_col(const EnergyArgs a) {
  constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int C = a.C;
  const int c = threadIdx.x % C, t = threadIdx.x / C;
  const int comp = blockIdx.y, inst = blockIdx.z;
  const int ix = blockIdx.x * C + c;
  const cx<T> *col = reinterpret_cast<const cx<T> *>(a.scratch) + ((long)inst * 2 + comp) * (long)N * a.nx + ix;
  const ColAcc<T> acc{reinterpret_cast<cx<T> *>(smem_raw), C, c};
  cx<T> v[1][E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[0][m] = col[(long)(t + m * TT) * a.nx];
  block_fft<LOGN, LOGE, -1, 1>(v, t, a.twy, acc);
  const double kL = a.gpar[4 * inst + 3];
  const double kx = a.dkx * kbin(ix, a.nx);
  const double shift = (comp == 0 ? -kL : kL) * kx;
  double s[1] = {0.0};
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const double ky = a.dky * kbin(t + m * TT, N);
    const double re = v[0][m].re, im = v[0][m].im;
    s[0] += (0.5 * (kx * kx + ky * ky) + shift) * (re * re + im * im);
  }
  block_sum<1>(s);
  if (threadIdx.x == 0) a.partials[((long)inst * 2 + comp) * gridDim.x + blockIdx.x] = s[0];
}

// ---------------------------------------------------- generic reductions

template <class T>
__global__ void __launch_bounds__(256) norm_kernel(const cx<T> *__restrict__ psi, long plane,
                                                   double *__restrict__ partials) {
  const int inst = blockIdx.y;
  const cx<T> *u = psi + (long)inst * 2 * plane, *d = u + plane;
  double s[2] = {0.0, 0.0};
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (long)gridDim.x * blockDim.x) {
    const cx<T> a = u[i], b = d[i];
    s[0] += double(a.re) * a.re + double(a.im) * a.im;
    s[1] += double(b.re) * b.re + double(b.im) * b.im;
  }
  block_sum<2>(s);
  if (threadIdx.x == 0) {
    partials[((long)inst * gridDim.x + blockIdx.x) * 2] = s[0];
    partials[((long)inst * gridDim.x + blockIdx.x) * 2 + 1] = s[1];
  }
}

template <class T>
__global__ void __launch_bounds__(256) residual_kernel(const cx<T> *__restrict__ psi, const cx<T> *__restrict__ prev,
                                                       long plane, double *__restrict__ partials) {
  const int inst = blockIdx.y;
  const long base = (long)inst * 2 * plane;
  double s[2] = {0.0, 0.0};
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * plane; i += (long)gridDim.x * blockDim.x) {
    const cx<T> a = psi[base + i], b = prev[base + i];
    const double dr = double(a.re) - b.re, di = double(a.im) - b.im;
    s[0] += dr * dr + di * di;
    s[1] += double(b.re) * b.re + double(b.im) * b.im;
  }
  block_sum<2>(s);
  if (threadIdx.x == 0) {
    partials[((long)inst * gridDim.x + blockIdx.x) * 2] = s[0];
    partials[((long)inst * gridDim.x + blockIdx.x) * 2 + 1] = s[1];
  }
}

// ------------------------------------------- comparator elementwise kernels

// R(tau) = X D X at every point, as one separate Hadamard-style pass.
template <class T, bool IMAG>
__global__ void __launch_bounds__(256) ref_R_kernel(const RowArgs a) {
  const long plane = (long)a.ny * a.nx;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int inst = blockIdx.y;
  if (i >= plane) return;
  const int y = int(i / a.nx), x = int(i - (long)y * a.nx);
  cx<T> *u = reinterpret_cast<cx<T> *>(a.psi) + (long)inst * 2 * plane + i;
  cx<T> *d = u + plane;
  const q4<T> px = reinterpret_cast<const q4<T> *>(a.tabx)[(long)inst * a.nx + x];
  const q4<T> ty = reinterpret_cast<const q4<T> *>(a.taby)[(long)inst * a.ny + y];
  T htau, xang;
  if constexpr (sizeof(T) == 4) { htau = a.htau_f; xang = a.xang_f; } else { htau = a.htau_d; xang = a.xang; }
  T vu, vd, q2z = T(0);
  if constexpr (IMAG) {
    vu = px.x * ty.x;
    vd = px.y * ty.y;
  } else {
    vu = px.x + ty.x;
    vd = px.y + ty.y;
  }
  const bool has2d = a.pot2d != nullptr;
  if (has2d) {
    const q4<T> q = reinterpret_cast<const q4<T> *>(a.pot2d)[i];
    if constexpr (IMAG) {
      vu *= exp(htau * q.x);
      vd *= exp(htau * q.y);
    } else {
      vu = d_fma(htau, q.x, vu);
      vd = d_fma(htau, q.y, vd);
    }
    q2z = q.z;
  }
  const XPoint<T> xc = xpoint<IMAG, T>(px, ty, has2d, q2z, xang);
  const int pieces = (a.omega_pieces & 3) | (has2d ? 4 : 0);
  const T *gp = reinterpret_cast<const T *>(a.gparT) + 4 * inst;
  cx<T> U = *u, D = *d;
  applyX<IMAG>(U, D, xc, pieces);
  opD<IMAG>(U, D, vu, vd, htau * gp[0], htau * gp[1], htau * gp[2]);
  applyX<IMAG>(U, D, xc, pieces);
  *u = U;
  *d = D;
}

// K(dt) with 1/(nx ny) on the transformed planes, as one separate pass.
template <class T>
__global__ void __launch_bounds__(256) ref_K_kernel(const ColArgs a) {
  const long plane = (long)a.ny * a.nx;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int pc = blockIdx.y;  // inst * 2 + comp
  if (i >= plane) return;
  const int ky = int(i / a.nx), kx = int(i - (long)ky * a.nx);
  cx<T> *p = reinterpret_cast<cx<T> *>(a.psi) + (long)pc * plane + i;
  const cx<T> am = reinterpret_cast<const cx<T> *>(a.kxt)[(long)pc * a.nx + kx];
  const cx<T> b = reinterpret_cast<const cx<T> *>(a.kyt)[ky];
  const cx<T> k1 = {d_fma(am.re, b.re, d_fma(-am.im, b.im, am.re + b.re)),
                    d_fma(am.re, b.im, d_fma(am.im, b.re, am.im + b.im))};
  const T inv = T(1) / T(plane);
  const cx<T> z = add_mul1(*p, k1);
  *p = {z.re * inv, z.im * inv};
}

}  // namespace spgpe
