// Kernels of the Fourier neural operator (FNO) used as the ground-state warm
// start: strided batched real and complex GEMMs (the pointwise channel maps,
// the truncated DFTs as contractions with twiddle matrices, the per-mode
// channel mixing, and all their transposes for the backward pass), split-K
// weight gradients with a fixed-order reduction, GELU, bias sums, the loss,
// and Adam with bfloat16 rounding of the weights used in the products.
//
// All products accumulate in FP32; weights are read as bfloat16.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "fno_internal.h"

namespace spgpe {
namespace fno {

namespace {

constexpr int TM = 64, TN = 64, TK = 16;  // output tile and K step of the GEMMs

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// C[bt](m, n) = alpha sum_k A[bt](m, k) B[bt](k, n) + beta C[bt](m, n) + bias[m],
// element (m, k) of A at A + bt sAb + m sAm + k sAk (likewise B, C).
// gridDim.z = batch * splits: split s of batch entry b covers k in
// [s ks, (s+1) ks); with `partial`, it writes its partial product to
// C + (b splits + s) sCs (alpha 1, beta and bias ignored; reduce_splits sums
// the batch * splits partials).
template <class TA>
__global__ void __launch_bounds__(256) gemm_r(int M, int N, int K, int splits, int partial, float alpha,
                                              const TA *__restrict__ A,
                                              long sAm, long sAk, long sAb, const float *__restrict__ B, long sBk,
                                              long sBn, long sBb, float beta, float *C, long sCm, long sCn, long sCb,
                                              long sCs, const float *__restrict__ bias) {
  __shared__ float As[TK][TM + 4];
  __shared__ float Bs[TK][TN + 4];
  const int bt = blockIdx.z / splits, sp = blockIdx.z - bt * splits;
  const int ks = (K + splits - 1) / splits, k0 = sp * ks, k1 = min(K, k0 + ks);
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  A += bt * sAb;
  B += bt * sBb;
  float acc[4][4] = {};
  for (int kk = k0; kk < k1; kk += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      const int mm = e / TK, k = e - mm * TK;  // k fastest: unit-stride A rows load coalesced
      const int gm = m0 + mm, gk = kk + k;
      As[k][mm] = (gm < M && gk < k1) ? to_f(A[gm * sAm + gk * sAk]) : 0.f;
    }
    for (int e = threadIdx.x; e < TN * TK; e += 256) {
      const int k = e / TN, nn = e - k * TN;
      const int gn = n0 + nn, gk = kk + k;
      Bs[k][nn] = (gn < N && gk < k1) ? B[gk * sBk + gn * sBn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *Cb = partial ? C + ((long)bt * splits + sp) * sCs : C + bt * sCb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float *c = Cb + gm * sCm + gn * sCn;
      if (partial) {
        *c = acc[i][j];
      } else {
        float v = alpha * acc[i][j];
        if (beta != 0.f) v = fmaf(beta, *c, v);
        if (bias) v += bias[gm];
        *c = v;
      }
    }
  }
}

// The same product for large M and N: BM x 128 output tiles (BM = 64 or
// 128), k steps of 8, each of the 256 threads accumulating (BM/16) x 8
// outputs in registers: rows ty*R + i and (BM/2) + ty*R + i (R = BM/32),
// columns tx*4 + j and 64 + tx*4 + j, so that the operand reads from shared
// memory are float2/float4s that hit every bank once.  Same arguments and
// split-K behaviour as gemm_r.
template <class TA, int BM>
__global__ void __launch_bounds__(256) gemm_r2(int M, int N, int K, int splits, int partial, float alpha,
                                               const TA *__restrict__ A, long sAm, long sAk, long sAb,
                                               const float *__restrict__ B, long sBk, long sBn, long sBb, float beta,
                                               float *C, long sCm, long sCn, long sCb, long sCs,
                                               const float *__restrict__ bias) {
  constexpr int BN = 128, BK = 8, R = BM / 32;  // R rows per half of the thread's rows
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  const int bt = blockIdx.z / splits, sp = blockIdx.z - bt * splits;
  const int ks = (K + splits - 1) / splits, k0 = sp * ks, k1 = min(K, k0 + ks);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  A += bt * sAb;
  B += bt * sBb;
  float acc[2 * R][8];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  // tile loads walk along whichever index has unit stride (full sectors)
  const bool a_m_fast = sAm == 1, b_k_fast = sBk == 1;
  for (int kk = k0; kk < k1; kk += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int mm, k;
      if (a_m_fast) {
        k = e / BM;
        mm = e - k * BM;
      } else {
        mm = e / BK;
        k = e - mm * BK;
      }
      const int gm = m0 + mm, gk = kk + k;
      As[k][mm] = (gm < M && gk < k1) ? to_f(A[gm * sAm + gk * sAk]) : 0.f;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      int nn, k;
      if (b_k_fast) {
        nn = e / BK;
        k = e - nn * BK;
      } else {
        k = e / BN;
        nn = e - k * BN;
      }
      const int gn = n0 + nn, gk = kk + k;
      Bs[k][nn] = (gn < N && gk < k1) ? B[gk * sBk + gn * sBn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[2 * R], b[8];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if constexpr (R == 4) {
          const float4 v = *reinterpret_cast<const float4 *>(&As[k][h * (BM / 2) + ty * R]);
          a[h * R] = v.x;
          a[h * R + 1] = v.y;
          a[h * R + 2] = v.z;
          a[h * R + 3] = v.w;
        } else {
          static_assert(R == 2, "BM is 64 or 128");
          const float2 v = *reinterpret_cast<const float2 *>(&As[k][h * (BM / 2) + ty * R]);
          a[h * R] = v.x;
          a[h * R + 1] = v.y;
        }
      }
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[k][64 + tx * 4]);
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 2 * R; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *Cb = partial ? C + ((long)bt * splits + sp) * sCs : C + bt * sCb;
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) {
    const int gm = m0 + (i / R) * (BM / 2) + ty * R + (i % R);
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = n0 + (j / 4) * 64 + tx * 4 + (j % 4);
      if (gn >= N) continue;
      float *c = Cb + gm * sCm + gn * sCn;
      if (partial) {
        *c = acc[i][j];
      } else {
        float v = alpha * acc[i][j];
        if (beta != 0.f) v = fmaf(beta, *c, v);
        if (bias) v += bias[gm];
        *c = v;
      }
    }
  }
}

// out[i] (+)= sum_s part[s][i] in the order s = 0, 1, ...
__global__ void reduce_splits(const float *__restrict__ part, long n, int splits, float *out, int accumulate) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float s = accumulate ? out[i] : 0.f;
    for (int k = 0; k < splits; ++k) s += part[(long)k * n + i];
    out[i] = s;
  }
}

struct c2 {
  float x, y;
};
__device__ __forceinline__ c2 ld_c(const float2 *p) { const float2 v = *p; return {v.x, v.y}; }
__device__ __forceinline__ c2 ld_c(const __nv_bfloat162 *p) {
  const __nv_bfloat162 v = *p;
  return {__low2float(v), __high2float(v)};
}

// Complex version of gemm_r (no splits, no bias): strides in complex elements;
// CA / CB conjugate the A / B operand.
template <class TA, bool CA, bool CB>
__global__ void __launch_bounds__(256) gemm_c(int M, int N, int K, const TA *__restrict__ A, long sAm, long sAk,
                                              long sAb, const float2 *__restrict__ B, long sBk, long sBn, long sBb,
                                              float beta, float2 *C, long sCm, long sCn, long sCb) {
  __shared__ c2 As[TK][TM + 1];
  __shared__ c2 Bs[TK][TN + 1];
  const int bt = blockIdx.z;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  A += bt * sAb;
  B += bt * sBb;
  C += bt * sCb;
  c2 acc[4][4] = {};
  for (int kk = 0; kk < K; kk += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      const int mm = e / TK, k = e - mm * TK;
      const int gm = m0 + mm, gk = kk + k;
      c2 v = {0.f, 0.f};
      if (gm < M && gk < K) v = ld_c(A + gm * sAm + gk * sAk);
      if (CA) v.y = -v.y;
      As[k][mm] = v;
    }
    for (int e = threadIdx.x; e < TN * TK; e += 256) {
      const int k = e / TN, nn = e - k * TN;
      const int gn = n0 + nn, gk = kk + k;
      c2 v = {0.f, 0.f};
      if (gn < N && gk < K) v = ld_c(B + gk * sBk + gn * sBn);
      if (CB) v.y = -v.y;
      Bs[k][nn] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < TK; ++k) {
      c2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float2 *c = C + gm * sCm + gn * sCn;
      float2 v = make_float2(acc[i][j].x, acc[i][j].y);
      if (beta != 0.f) {
        const float2 o = *c;
        v.x = fmaf(beta, o.x, v.x);
        v.y = fmaf(beta, o.y, v.y);
      }
      *c = v;
    }
  }
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

__global__ void gelu_fwd(const float *__restrict__ u, float *__restrict__ v, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    v[i] = gelu_f(u[i]);
}

__global__ void gelu_bwd(const float *__restrict__ u, float *__restrict__ d, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    d[i] *= gelu_d(u[i]);
}

// grad[c] (+)= sum over samples b and points p of x[b][c][p] (fixed order).
// Bias gradient grad[c] += sum_b sum_p x[b][c][p], in two stages: kBiasSlices
// blocks per channel each sum a contiguous slice of the points (float32 per
// thread over at most a few dozen values, then a fixed tree), and one block
// adds the slices of every channel in a fixed order in FP64.
constexpr int kBiasSlices = 64;

__global__ void __launch_bounds__(256) bias_grad_slices(const float *__restrict__ x, int B, int C, long P,
                                                        double *part) {
  const int c = blockIdx.x / kBiasSlices, sl = blockIdx.x - c * kBiasSlices;
  const long n = (long)B * P, per = (n + kBiasSlices - 1) / kBiasSlices;
  const long i0 = sl * per, i1 = min(n, i0 + per);
  float s = 0.f;
  for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const long b = i / P, p = i - b * P;
    s += x[(b * C + c) * P + p];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void bias_grad_sum(const double *__restrict__ part, int C, float *grad) {
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double t = 0.0;
    for (int sl = 0; sl < kBiasSlices; ++sl) t += part[(long)c * kBiasSlices + sl];
    grad[c] += (float)t;
  }
}

// Per sample: num = sum (out - t)^2, den = sum t^2 into sums[b][2], in two
// stages like the bias gradient: kBiasSlices blocks per sample sum a slice
// (float32 per thread, a fixed tree, FP64 across warps) into part[b][slice][2],
// then one thread per sample adds the slices in a fixed order in FP64.
__global__ void __launch_bounds__(256) loss_slices(const float *__restrict__ out, const float *__restrict__ t, long n,
                                                   double *part) {
  const int b = blockIdx.x / kBiasSlices, sl = blockIdx.x - b * kBiasSlices;
  const long per = (n + kBiasSlices - 1) / kBiasSlices, i0 = sl * per, i1 = min(n, i0 + per);
  float num = 0.f, den = 0.f;
  for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const float o = out[(long)b * n + i], tv = t[(long)b * n + i], d = o - tv;
    num = fmaf(d, d, num);
    den = fmaf(tv, tv, den);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  __shared__ float r0[8], r1[8];
  if ((threadIdx.x & 31) == 0) {
    r0[threadIdx.x >> 5] = num;
    r1[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += r0[w];
      c += r1[w];
    }
    part[2 * (long)blockIdx.x] = a;
    part[2 * (long)blockIdx.x + 1] = c;
  }
}

__global__ void loss_sum(const double *__restrict__ part, int B, double *sums) {
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    double a = 0.0, c = 0.0;
    for (int sl = 0; sl < kBiasSlices; ++sl) {
      a += part[2 * ((long)b * kBiasSlices + sl)];
      c += part[2 * ((long)b * kBiasSlices + sl) + 1];
    }
    sums[2 * b] = a;
    sums[2 * b + 1] = c;
  }
}

// dout = 2 (out - t) / den_b / B.
__global__ void loss_grad(const float *__restrict__ out, const float *__restrict__ t, long n, int B,
                          const double *__restrict__ sums, float *dout) {
  const long total = n * B;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int b = (int)(i / n);
    dout[i] = (float)(2.0 * ((double)out[i] - (double)t[i]) / sums[2 * b + 1] / B);
  }
}

// Adam (Kingma & Ba 2015) with bias correction on the FP32 master weights;
// the bfloat16 weights used in the products are the rounded masters.
__global__ void adam(float *w, __nv_bfloat16 *wb, float *wr, const float *__restrict__ g, float *m, float *v, long n,
                     float lr, float c1, float c2) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(0.9f, m[i], 0.1f * gi), vi = fmaf(0.999f, v[i], 0.001f * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    w[i] = wi;
    const __nv_bfloat16 r = __float2bfloat16_rn(wi);
    wb[i] = r;
    wr[i] = __bfloat162float(r);
  }
}

__global__ void to_bf16(const float *__restrict__ w, __nv_bfloat16 *wb, float *wr, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const __nv_bfloat16 r = __float2bfloat16_rn(w[i]);
    wb[i] = r;
    wr[i] = __bfloat162float(r);
  }
}

int grid_for(long n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

}  // namespace

cudaError_t gemm_real(const GemmR &g, cudaStream_t st) {
  // the pointwise channel maps with bfloat16 weights: tensor cores
  if (gemm_tc_applies(g)) return gemm_real_tc(g, st);
  // large products: the register-tiled kernel (BM = 128, or 64 when M is small)
  if (g.N >= 128 && g.M >= 64) {
    const int bm = g.M >= 128 ? 128 : 64;
    const dim3 grid((g.N + 127) / 128, (g.M + bm - 1) / bm, g.batch * g.splits);
#define SPGPE_R2(TA, BMV)                                                                                           \
  gemm_r2<TA, BMV><<<grid, 256, 0, st>>>(g.M, g.N, g.K, g.splits, g.partial ? 1 : 0, g.alpha,                     \
                                         static_cast<const TA *>(g.A), g.sAm, g.sAk, g.sAb, g.B, g.sBk, g.sBn,     \
                                         g.sBb, g.beta, g.C, g.sCm, g.sCn, g.sCb, g.sCs, g.bias)
    if (g.a_bf16) {
      if (bm == 128) SPGPE_R2(__nv_bfloat16, 128);
      else SPGPE_R2(__nv_bfloat16, 64);
    } else {
      if (bm == 128) SPGPE_R2(float, 128);
      else SPGPE_R2(float, 64);
    }
#undef SPGPE_R2
    return cudaGetLastError();
  }
  const dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, g.batch * g.splits);
  if (g.a_bf16)
    gemm_r<__nv_bfloat16><<<grid, 256, 0, st>>>(g.M, g.N, g.K, g.splits, g.partial ? 1 : 0, g.alpha,
                                                 static_cast<const __nv_bfloat16 *>(g.A), g.sAm, g.sAk, g.sAb, g.B,
                                                 g.sBk, g.sBn, g.sBb, g.beta, g.C, g.sCm, g.sCn, g.sCb, g.sCs, g.bias);
  else
    gemm_r<float><<<grid, 256, 0, st>>>(g.M, g.N, g.K, g.splits, g.partial ? 1 : 0, g.alpha,
                                        static_cast<const float *>(g.A), g.sAm, g.sAk, g.sAb, g.B, g.sBk, g.sBn,
                                        g.sBb, g.beta, g.C, g.sCm, g.sCn, g.sCb, g.sCs, g.bias);
  return cudaGetLastError();
}

cudaError_t sum_splits(const float *part, long n, int splits, float *out, bool accumulate, cudaStream_t st) {
  reduce_splits<<<grid_for(n), 256, 0, st>>>(part, n, splits, out, accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t gemm_complex(const GemmC &g, cudaStream_t st) {
  const dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, g.batch);
#define SPGPE_GC(TA, CA, CB)                                                                                    \
  gemm_c<TA, CA, CB><<<grid, 256, 0, st>>>(g.M, g.N, g.K, static_cast<const TA *>(g.A), g.sAm, g.sAk, g.sAb, g.B, \
                                           g.sBk, g.sBn, g.sBb, g.beta, g.C, g.sCm, g.sCn, g.sCb)
  if (g.a_bf16) {
    if (g.conj_a) SPGPE_GC(__nv_bfloat162, true, false);
    else SPGPE_GC(__nv_bfloat162, false, false);
  } else if (g.conj_a) {
    SPGPE_GC(float2, true, false);
  } else if (g.conj_b) {
    SPGPE_GC(float2, false, true);
  } else {
    SPGPE_GC(float2, false, false);
  }
#undef SPGPE_GC
  return cudaGetLastError();
}

cudaError_t gelu_forward(const float *u, float *v, long n, cudaStream_t st) {
  gelu_fwd<<<grid_for(n), 256, 0, st>>>(u, v, n);
  return cudaGetLastError();
}

cudaError_t gelu_backward(const float *u, float *d, long n, cudaStream_t st) {
  gelu_bwd<<<grid_for(n), 256, 0, st>>>(u, d, n);
  return cudaGetLastError();
}

cudaError_t bias_gradient(const float *x, int B, int C, long P, float *grad, double *scratch, cudaStream_t st) {
  bias_grad_slices<<<C * kBiasSlices, 256, 0, st>>>(x, B, C, P, scratch);
  bias_grad_sum<<<1, 256, 0, st>>>(scratch, C, grad);
  return cudaGetLastError();
}

cudaError_t loss_terms(const float *out, const float *t, long n, int B, double *sums, float *dout, cudaStream_t st) {
  double *part = sums + 2 * (long)B;
  loss_slices<<<B * kBiasSlices, 256, 0, st>>>(out, t, n, part);
  loss_sum<<<1, 256, 0, st>>>(part, B, sums);
  if (dout) loss_grad<<<grid_for(n * B), 256, 0, st>>>(out, t, n, B, sums, dout);
  return cudaGetLastError();
}

cudaError_t adam_update(float *w, void *wb, float *wr, const float *g, float *m, float *v, long n, float lr, int t,
                        cudaStream_t st) {
  const float c1 = (float)(1.0 - std::pow(0.9, t)), c2 = (float)(1.0 - std::pow(0.999, t));
  adam<<<grid_for(n), 256, 0, st>>>(w, static_cast<__nv_bfloat16 *>(wb), wr, g, m, v, n, lr, c1, c2);
  return cudaGetLastError();
}

cudaError_t round_weights(const float *w, void *wb, float *wr, long n, cudaStream_t st) {
  to_bf16<<<grid_for(n), 256, 0, st>>>(w, static_cast<__nv_bfloat16 *>(wb), wr, n);
  return cudaGetLastError();
}

}  // namespace fno
}  // namespace spgpe
