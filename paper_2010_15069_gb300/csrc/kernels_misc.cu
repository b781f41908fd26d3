// Precision conversion of spinors (the complex64 / complex128 ladder of
// spgpe_relax): round complex128 to complex64, or widen complex64 exactly.
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

}  // namespace spgpe
