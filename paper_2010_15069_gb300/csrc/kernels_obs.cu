// Observables of the spin-Hall ground states (Sec. 6) and the annealing noise
// of the ground-state protocol, both precisions.
//
//  * obs_sums: FP64 sums rho_up rho_dn, rho_up^2, rho_dn^2 and rho_up + rho_dn
//    per instance (the phase-separation parameter of Eq. 14 and the total).
//  * radial_hist: atom number in radial bins of width h about the trap centre
//    (the contour of Eq. 15 encloses 99 % of it).
//  * winding: phase steps of psi_j (bilinearly interpolated) around the circle
//    of radius R99, summed in FP64 (Eq. 15 winding numbers).
//  * add_noise: psi += sigma xi, xi complex standard normal from a
//    counter-based SplitMix64 stream (Sec. 6 annealing).
#include <cuda_runtime.h>

#include "fft_core.cuh"
#include "internal.h"

namespace spgpe {

namespace {

template <int K> __device__ __forceinline__ void obs_block_sum(double (&v)[K]) {
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

template <class T>
__global__ void __launch_bounds__(256) obs_sums(const cx<T> *__restrict__ psi, long plane, double *partials) {
  const int inst = blockIdx.y;
  const cx<T> *u = psi + (long)inst * 2 * plane, *d = u + plane;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (long)gridDim.x * blockDim.x) {
    const cx<T> a = u[i], b = d[i];
    const double ru = double(a.re) * a.re + double(a.im) * a.im;
    const double rd = double(b.re) * b.re + double(b.im) * b.im;
    s[0] += ru * rd;
    s[1] += ru * ru;
    s[2] += rd * rd;
    s[3] += ru + rd;
  }
  obs_block_sum<4>(s);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) partials[((long)inst * gridDim.x + blockIdx.x) * 4 + k] = s[k];
}

// One block per (row group, instance): a shared-memory histogram of nb bins,
// merged into hist[inst][nb] (zeroed by the caller).
template <class T>
__global__ void __launch_bounds__(256) radial_hist(const cx<T> *__restrict__ psi, ObsGeom g, int rows_per_block,
                                                   double *hist) {
  extern __shared__ double sh[];
  const int inst = blockIdx.y;
  for (int b = threadIdx.x; b < g.nb; b += blockDim.x) sh[b] = 0.0;
  __syncthreads();
  const long plane = (long)g.nx * g.ny;
  const cx<T> *u = psi + (long)inst * 2 * plane, *d = u + plane;
  const int y0 = blockIdx.x * rows_per_block;
  const int y1 = min(g.ny, y0 + rows_per_block);
  for (long i = (long)y0 * g.nx + threadIdx.x; i < (long)y1 * g.nx; i += blockDim.x) {
    const int iy = (int)(i / g.nx), ix = (int)(i - (long)iy * g.nx);
    const double x = -g.xmax + ix * g.dx, y = -g.ymax + iy * g.dy;
    const int bin = min(g.nb - 1, (int)(sqrt(x * x + y * y) / g.h));
    const cx<T> a = u[i], b = d[i];
    atomicAdd(&sh[bin], double(a.re) * a.re + double(a.im) * a.im + double(b.re) * b.re + double(b.im) * b.im);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < g.nb; b += blockDim.x)
    if (sh[b] != 0.0) atomicAdd(&hist[(long)inst * g.nb + b], sh[b]);
}

template <class T> __device__ __forceinline__ double phase_at(const cx<T> *f, const ObsGeom &g, double x, double y) {
  const double uu = (x + g.xmax) / g.dx, vv = (y + g.ymax) / g.dy;
  const double fu0 = floor(uu), fv0 = floor(vv);
  const double fu = uu - fu0, fv = vv - fv0;
  const int i0 = (((int)fu0) % g.nx + g.nx) % g.nx, j0 = (((int)fv0) % g.ny + g.ny) % g.ny;
  const int i1 = (i0 + 1) % g.nx, j1 = (j0 + 1) % g.ny;
  const cx<T> a = f[(long)j0 * g.nx + i0], b = f[(long)j0 * g.nx + i1];
  const cx<T> c = f[(long)j1 * g.nx + i0], e = f[(long)j1 * g.nx + i1];
  const double w00 = (1 - fu) * (1 - fv), w10 = fu * (1 - fv), w01 = (1 - fu) * fv, w11 = fu * fv;
  const double re = w00 * a.re + w10 * b.re + w01 * c.re + w11 * e.re;
  const double im = w00 * a.im + w10 * b.im + w01 * c.im + w11 * e.im;
  return atan2(im, re);
}

// One block per (component, instance): sum of the wrapped phase steps around
// the circle of radius R[inst] with npts points; out[inst][comp] = n.
template <class T>
__global__ void __launch_bounds__(256) winding(const cx<T> *__restrict__ psi, ObsGeom g, const double *R, int npts,
                                               double *out) {
  const int comp = blockIdx.x, inst = blockIdx.y;
  const long plane = (long)g.nx * g.ny;
  const cx<T> *f = psi + ((long)inst * 2 + comp) * plane;
  const double r = R[inst];
  double s[1] = {0.0};
  for (int k = threadIdx.x; k < npts; k += blockDim.x) {
    double s0, c0, s1, c1;
    sincospi(2.0 * k / npts, &s0, &c0);
    sincospi(2.0 * ((k + 1) % npts) / npts, &s1, &c1);
    double dph = phase_at(f, g, r * c1, r * s1) - phase_at(f, g, r * c0, r * s0);
    const double pi = 3.14159265358979323846;
    while (dph > pi) dph -= 2.0 * pi;
    while (dph <= -pi) dph += 2.0 * pi;
    s[0] += dph;
  }
  obs_block_sum<1>(s);
  if (threadIdx.x == 0) out[(long)inst * 2 + comp] = rint(s[0] / (2.0 * 3.14159265358979323846));
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based generator:
// draw c of stream `seed` is the output function applied to
// seed + (c + 1) * 0x9E3779B97F4A7C15.
__device__ __forceinline__ unsigned long long mix64(unsigned long long seed, unsigned long long c) {
  unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// psi += sigma xi: element e of instance i (global index inst0 + i) takes the
// draws 2E and 2E + 1, E = (inst0 + i) * n2 + e, as uniforms u = (draw >> 11)
// 2^-53, and xi = sqrt(-ln(1 - u1)) e^{2 pi i u2}.
template <class T>
__global__ void __launch_bounds__(256) add_noise(cx<T> *psi, long n2, int ninst, long inst0, double sigma,
                                                 unsigned long long seed) {
  const long total = n2 * ninst;
  for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < total; j += (long)gridDim.x * blockDim.x) {
    const unsigned long long E = (unsigned long long)(inst0 * n2 + j);
    const double u1 = (double)(mix64(seed, 2 * E) >> 11) * 0x1.0p-53;
    const double u2 = (double)(mix64(seed, 2 * E + 1) >> 11) * 0x1.0p-53;
    const double r = sigma * sqrt(-log(1.0 - u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    cx<T> v = psi[j];
    v.re = T(double(v.re) + r * cs);
    v.im = T(double(v.im) + r * sn);
    psi[j] = v;
  }
}

template <class T> cudaError_t obs_launch(const void *psi, const ObsGeom &g, int ninst, double *partials,
                                          int sum_blocks, double *hist, const double *R, int npts, double *wind,
                                          int phase, cudaStream_t st) {
  const cx<T> *p = reinterpret_cast<const cx<T> *>(psi);
  if (phase == 0) {
    obs_sums<T><<<dim3(sum_blocks, ninst), 256, 0, st>>>(p, (long)g.nx * g.ny, partials);
    const int rpb = (g.ny + 63) / 64;  // 64 row groups per instance
    const size_t sm = (size_t)g.nb * sizeof(double);
    if (sm > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(radial_hist<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    radial_hist<T><<<dim3((g.ny + rpb - 1) / rpb, ninst), 256, sm, st>>>(p, g, rpb, hist);
  } else {
    winding<T><<<dim3(2, ninst), 256, 0, st>>>(p, g, R, npts, wind);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_observables(int es, const void *psi, const ObsGeom &g, int ninst, double *partials,
                               int sum_blocks, double *hist, const double *R, int npts, double *wind, int phase,
                               cudaStream_t st) {
  return es == 8 ? obs_launch<float>(psi, g, ninst, partials, sum_blocks, hist, R, npts, wind, phase, st)
                 : obs_launch<double>(psi, g, ninst, partials, sum_blocks, hist, R, npts, wind, phase, st);
}

cudaError_t launch_add_noise(int es, void *psi, long n2, int ninst, long inst0, double sigma, unsigned long long seed,
                             int sms, cudaStream_t st) {
  const long want = (n2 * ninst + 255) / 256;
  const int grid = (int)(want < 8L * sms ? want : 8L * sms);
  if (grid < 1) return cudaSuccess;
  if (es == 8)
    add_noise<float><<<grid, 256, 0, st>>>(reinterpret_cast<cx<float> *>(psi), n2, ninst, inst0, sigma, seed);
  else
    add_noise<double><<<grid, 256, 0, st>>>(reinterpret_cast<cx<double> *>(psi), n2, ninst, inst0, sigma, seed);
  return cudaGetLastError();
}

}  // namespace spgpe
