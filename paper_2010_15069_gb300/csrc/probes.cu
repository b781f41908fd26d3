// Microbenchmarks of the ceilings the kernels are measured against: FP32 and
// FP64 fused multiply-add throughput, sincosf throughput, read bandwidth over
// working sets from a few MB to well above the L2 size (the bandwidth step
// shows the L2 capacity), and the HBM copy bandwidth.  They only launch
// kernels on a stream of their own and change no device setting; timings are
// CUDA events around each launch after a warm-up launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "spgpe.h"

namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

// x <- x a + b on kChains independent chains, `iters` times.  The result is
// written only when it equals an impossible value, so nothing is elided.
template <class T> __global__ void __launch_bounds__(256) fma_kernel(T *sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = T(threadIdx.x) * T(1e-3) + T(k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == T(-12345.0)) sink[blockIdx.x] = s;
}

// Four independent chains of sincosf on arguments in [0, 1].
__global__ void __launch_bounds__(256) sincos_kernel(float *sink, int iters) {
  float x[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) x[k] = 0.25f * k + 1e-4f * threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s, c;
      sincosf(x[k], &s, &c);
      x[k] = fmaf(0.5f, s, 0.25f * c);  // stays in [0, 1]
    }
  }
  const float t = x[0] + x[1] + x[2] + x[3];
  if (t == -12345.f) sink[blockIdx.x] = t;
}

// Read n float4 `reps` times (grid-stride), summing them.
__global__ void __launch_bounds__(256) read_kernel(const float4 *__restrict__ p, long n, int reps, float *sink) {
  float acc = 0.f;
  const long stride = (long)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const float4 v = __ldcg(p + i);
      acc += v.x + v.y + v.z + v.w;
    }
  if (acc == -12345.f) sink[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) copy_kernel(const float4 *__restrict__ a, float4 *__restrict__ b, long n) {
  const long stride = (long)gridDim.x * blockDim.x;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) b[i] = a[i];
}

// Time launch() after one untimed run; milliseconds (or -1 on error).
template <class F> float time_ms(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, F &&launch) {
  launch();
  if (cudaEventRecord(e0, s) != cudaSuccess) return -1.f;
  launch();
  if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
  if (cudaGetLastError() != cudaSuccess) return -1.f;
  float ms = -1.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

}  // namespace

extern "C" int spgpe_probe_ceilings(double *out, int n_out) {
  if (!out || n_out < SPGPE_PROBE_COUNT) return SPGPE_EINVAL;
  for (int i = 0; i < SPGPE_PROBE_COUNT; ++i) out[i] = NAN;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return SPGPE_ECUDA;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float *sink = nullptr;
  float4 *buf = nullptr;
  const long nbig = (1L << 30) / 16;  // 1 GiB of float4 (two halves for the copy)
  int rc = SPGPE_ECUDA;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&sink, 65536 * sizeof(float)) != cudaSuccess) {
    goto done;
  }
  if (cudaMalloc(&buf, nbig * sizeof(float4)) != cudaSuccess) {
    rc = SPGPE_ENOMEM;
    goto done;
  }
  if (cudaMemsetAsync(buf, 0, nbig * sizeof(float4), s) != cudaSuccess) goto done;
  {
    const int blocks = sms * 8, threads = 256;
    const double nthreads = (double)blocks * threads;
    // FP32 FMA: 2 flop each
    const int it32 = 16384;
    float ms = time_ms(s, e0, e1, [&] { fma_kernel<float><<<blocks, threads, 0, s>>>(sink, it32, 0.9999f, 1e-4f); });
    if (ms <= 0) goto done;
    out[0] = 2.0 * nthreads * kChains * it32 / (ms * 1e-3) / 1e12;
    // FP64 FMA
    const int it64 = 512;
    ms = time_ms(s, e0, e1, [&] { fma_kernel<double><<<blocks, threads, 0, s>>>(reinterpret_cast<double *>(sink), it64, 0.9999, 1e-4); });
    if (ms <= 0) goto done;
    out[1] = 2.0 * nthreads * kChains * it64 / (ms * 1e-3) / 1e12;
    // sincosf calls per second
    const int itsc = 2048;
    ms = time_ms(s, e0, e1, [&] { sincos_kernel<<<blocks, threads, 0, s>>>(sink, itsc); });
    if (ms <= 0) goto done;
    out[2] = nthreads * 4.0 * itsc / (ms * 1e-3) / 1e9;
    // read bandwidth over working sets of 16 ... 512 MiB (each read ~2 GiB in all)
    const int sizes_mb[SPGPE_PROBE_NSIZES] = {16, 32, 64, 96, 128, 160, 192, 256, 512};
    for (int k = 0; k < SPGPE_PROBE_NSIZES; ++k) {
      const long n = (long)sizes_mb[k] * (1L << 20) / 16;
      const int reps = (int)std::max(1L, (2L << 30) / (n * 16));
      ms = time_ms(s, e0, e1, [&] { read_kernel<<<blocks, threads, 0, s>>>(buf, n, reps, sink); });
      if (ms <= 0) goto done;
      out[4 + k] = (double)n * 16 * reps / (ms * 1e-3) / 1e9;
    }
    // HBM copy: read 512 MiB and write 512 MiB
    ms = time_ms(s, e0, e1, [&] { copy_kernel<<<blocks, threads, 0, s>>>(buf, buf + nbig / 2, nbig / 2); });
    if (ms <= 0) goto done;
    out[3] = (double)nbig * 16 / (ms * 1e-3) / 1e9;
    rc = SPGPE_OK;
  }
done:
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaGetLastError();
  return rc;
}
