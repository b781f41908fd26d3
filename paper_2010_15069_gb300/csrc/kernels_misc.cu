// Precision conversion of spinors (the complex64 / complex128 ladder of
// spgpe_relax): round complex128 to complex64, or widen complex64 exactly.
// And the probe of the bounded-wait failure path.
#include "async_copy.cuh"
#include "internal.h"

namespace spgpe {

__global__ void __launch_bounds__(256) round_to_c64(const double2 *__restrict__ src, float2 *__restrict__ dst,
                                                    long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    dst[i] = make_float2((float)v.x, (float)v.y);
  }
}

__global__ void __launch_bounds__(256) widen_to_c128(const float2 *__restrict__ src, double2 *__restrict__ dst,
                                                     long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float2 v = src[i];
    dst[i] = make_double2((double)v.x, (double)v.y);
  }
}

cudaError_t launch_convert(const void *src, int src_es, void *dst, int dst_es, long n, int sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long want = (n + 255) / 256;
  const int grid = (int)(want < 8L * sms ? want : 8L * sms);
  if (src_es == 16 && dst_es == 8)
    round_to_c64<<<grid, 256, 0, s>>>(reinterpret_cast<const double2 *>(src), reinterpret_cast<float2 *>(dst), n);
  else if (src_es == 8 && dst_es == 16)
    widen_to_c128<<<grid, 256, 0, s>>>(reinterpret_cast<const float2 *>(src), reinterpret_cast<double2 *>(dst), n);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// Probe of the failure path the streaming passes take when a tile transfer
// never lands: one thread arms an mbarrier that nothing will ever complete
// (no copy is issued, no other thread arrives), waits on it with the given
// cycle budget, and on giving up sets the timeout bit in the context's error
// flags and returns, as the passes do.  Nothing is in flight when it leaves.
__global__ void wait_probe(int *flags, long long budget) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_fence_init();
  const long long t0 = clock64();
  bool done = false;
  while (!(done = mbar_try_wait(&bar, 0)) && clock64() - t0 <= budget) {
  }
  if (!done) atomicOr(flags, kErrTimeout);
}

cudaError_t launch_wait_probe(int *flags, long long budget, cudaStream_t s) {
  wait_probe<<<1, 32, 0, s>>>(flags, budget);
  return cudaGetLastError();
}

}  // namespace spgpe
