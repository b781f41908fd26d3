// Launchers of the Fourier-neural-operator kernels (fno_kernels.cu), used by
// the C ABI in fno.cu.
#pragma once
#include <cuda_runtime.h>

namespace spgpe {
namespace fno {

// C(m, n) = alpha sum_k A(m, k) B(k, n) + beta C(m, n) + bias[m] per batch
// entry; element (m, k) of A at A + b sAb + m sAm + k sAk (likewise B, C).
// partial: split-K over `splits` ranges of k, the partial product of split s
// of batch entry b to C + (b splits + s) sCs (alpha 1, beta and bias
// ignored) for sum_splits.
struct GemmR {
  int M, N, K, batch = 1, splits = 1;
  bool partial = false;
  float alpha = 1.f, beta = 0.f;
  const void *A;
  bool a_bf16 = false;
  long sAm, sAk, sAb = 0;
  const float *B;
  long sBk, sBn, sBb = 0;
  float *C;
  long sCm, sCn, sCb = 0, sCs = 0;
  const float *bias = nullptr;
  // device error flags of the model; non-null also admits the tensor-core
  // path (gemm_real_tc), which records a wait that ran out there
  int *flags = nullptr;
};

// Complex C(m, n) = sum_k op(A)(m, k) op(B)(k, n) + beta C(m, n), strides in
// complex elements; op conjugates when conj_a / conj_b (not both); A may be
// bfloat16 pairs (a_bf16; then not conjugated).
struct GemmC {
  int M, N, K, batch = 1;
  float beta = 0.f;
  const void *A;
  bool a_bf16 = false, conj_a = false, conj_b = false;
  long sAm, sAk, sAb = 0;
  const float2 *B;
  long sBk, sBn, sBb = 0;
  float2 *C;
  long sCm, sCn, sCb = 0;
};

cudaError_t gemm_real(const GemmR &g, cudaStream_t st);
// The same product on the tensor cores (fno_tc.cu) for the pointwise channel
// maps: bfloat16 weights A (sAb = 0; M = 64 or 128 rows, K = 64 or 128), a
// float32 B with unit stride along N (N a multiple of 128), C with unit
// stride along N, no split-K, alpha = 1, flags set; cudaErrorNotSupported
// for any other shape.
bool gemm_tc_applies(const GemmR &g);
cudaError_t gemm_real_tc(const GemmR &g, cudaStream_t st);
cudaError_t sum_splits(const float *part, long n, int splits, float *out, bool accumulate, cudaStream_t st);
cudaError_t gemm_complex(const GemmC &g, cudaStream_t st);
cudaError_t gelu_forward(const float *u, float *v, long n, cudaStream_t st);
cudaError_t gelu_backward(const float *u, float *d, long n, cudaStream_t st);
// grad[c] += sum over the batch and the points of x[b][c][p]; scratch holds
// 64 C doubles.
cudaError_t bias_gradient(const float *x, int B, int C, long P, float *grad, double *scratch, cudaStream_t st);
// sums[2 b], sums[2 b + 1] = sum (out - t)^2, sum t^2 of sample b; sums holds
// 130 B doubles (the rest is scratch); dout (nullable) = 2 (out - t) / den_b / B.
cudaError_t loss_terms(const float *out, const float *t, long n, int B, double *sums, float *dout, cudaStream_t st);
// Adam on the FP32 masters w; wb (bfloat16) and wr (FP32) receive the rounded weights.
cudaError_t adam_update(float *w, void *wb, float *wr, const float *g, float *m, float *v, long n, float lr, int t,
                        cudaStream_t st);
cudaError_t round_weights(const float *w, void *wb, float *wr, long n, cudaStream_t st);

}  // namespace fno
}  // namespace spgpe
