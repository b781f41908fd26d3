// spgpe_norm_noalloc: atom numbers of a spinor batch without allocating.
//
// The per-block partial sums and the per-instance totals live in a
// file-scope device array (kStaticDoubles doubles, 256 KiB) that every GPU
// loading this library holds until the process exits.  Host code must not
// use the array's name as a device address (it is a host-side stand-in); the
// device address is looked up with cudaGetSymbolAddress once per device and
// cached.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "spgpe.h"
#include "internal.h"
#include "kernels.cuh"

namespace {

constexpr int kBlocks = 64;              // partial sums per instance and component
constexpr int kPerInst = 2 * kBlocks + 2;
constexpr int kStaticDoubles = 32768;    // 256 KiB
constexpr int kMaxInst = kStaticDoubles / kPerInst;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_norm_scratch[kStaticDoubles];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Sum the kBlocks partials of each instance in a fixed order and scale by
// dx dy.  Layout of the scratch: partials [ninst][kBlocks][2], then totals
// [ninst][2].  Every slot read here was written by the preceding launch of the
// same call, so nothing needs clearing between calls.
__global__ void __launch_bounds__(64) norm_finish(double *scratch, int ninst, double w) {
  const int inst = blockIdx.x;
  double s[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < kBlocks; b += blockDim.x) {
    s[0] += scratch[((long)inst * kBlocks + b) * 2];
    s[1] += scratch[((long)inst * kBlocks + b) * 2 + 1];
  }
  spgpe::block_sum<2>(s);
  if (threadIdx.x == 0) {
    double *tot = scratch + (long)ninst * kBlocks * 2;
    tot[2 * inst] = s[0] * w;
    tot[2 * inst + 1] = s[1] * w;
  }
}

// Device address of the scratch array on the current device (set up once).
cudaError_t scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_norm_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = static_cast<double *>(g_addr[dev]);
  return cudaSuccess;
}

}  // namespace

extern "C" int spgpe_norm_noalloc(const void *psi, int nx, int ny, int ninst, double xmax, double ymax,
                                  int dtype, void *cuda_stream, double *out) {
  if (!psi || !out || nx < 1 || ny < 1 || ninst < 1 || (long)nx * ny > (1L << 30) ||
      !(std::isfinite(xmax) && xmax > 0 && std::isfinite(ymax) && ymax > 0) ||
      (dtype != SPGPE_C64 && dtype != SPGPE_C128))
    return SPGPE_EINVAL;
  if (ninst > kMaxInst) return SPGPE_EINVAL;  // beyond the static scratch
  double *scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return SPGPE_ECUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const long plane = (long)nx * ny;
  cudaError_t e = dtype == SPGPE_C64
                      ? spgpe::launch_norm<float>(psi, plane, ninst, scratch, kBlocks, st)
                      : spgpe::launch_norm<double>(psi, plane, ninst, scratch, kBlocks, st);
  if (e != cudaSuccess) return SPGPE_ECUDA;
  const double w = (2.0 * xmax / nx) * (2.0 * ymax / ny);
  norm_finish<<<ninst, 64, 0, st>>>(scratch, ninst, w);
  if (cudaGetLastError() != cudaSuccess) return SPGPE_ECUDA;
  if (cudaMemcpyAsync(out, scratch + (long)ninst * kBlocks * 2, (size_t)ninst * 2 * sizeof(double),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SPGPE_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPGPE_ECUDA;
  for (int i = 0; i < 2 * ninst; ++i)
    if (!std::isfinite(out[i])) return SPGPE_ENONFINITE;
  return SPGPE_OK;
}
