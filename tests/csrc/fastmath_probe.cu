// Test probe of the single-precision elementary functions of the pointwise
// operators (paper_2010_15069_gb300/csrc/fastmath.cuh): one thread per
// argument evaluates the selected function and writes its float results.
// Built by tests/test_fastmath_gpu.py; not part of the library.
#include <cuda_runtime.h>

#include "fastmath.cuh"

namespace {

// fn: 0 expi2_m1 -> (wre, wim); 1 expm1_f -> (e); 2 expm1_small -> (e);
// 3 shear_consts_2h (every tier, out of line) -> (t, s, neg);
// 4 shear_consts_2h_small -> (t, s); 5 shear_consts_2h_tiny -> (t, s);
// 6 expm1_quarter -> (e).
// out holds 3 floats per argument.
__global__ void probe(int fn, const float *__restrict__ x, int n, float *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float h = x[i];
  float a = 0.f, b = 0.f, c = 0.f;
  switch (fn) {
    case 0: spgpe::expi2_m1(h, a, b); break;
    case 1: a = spgpe::expm1_f(h); break;
    case 2: a = spgpe::expm1_small(h); break;
    case 3: {
      bool neg;
      spgpe::shear_consts_2h(h, a, b, neg);
      c = neg ? 1.f : 0.f;
      break;
    }
    case 4: spgpe::shear_consts_2h_small(h, a, b); break;
    case 6: a = spgpe::expm1_quarter(h); break;
    default: spgpe::shear_consts_2h_tiny(h, a, b); break;
  }
  out[3 * i] = a;
  out[3 * i + 1] = b;
  out[3 * i + 2] = c;
}

}  // namespace

// x and out are device pointers (n floats in, 3 n floats out); returns the
// CUDA status of the launch and of the synchronisation after it.
extern "C" int fastmath_probe(int fn, const float *x, int n, float *out) {
  if (n <= 0) return 0;
  probe<<<(n + 255) / 256, 256>>>(fn, x, n, out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}
