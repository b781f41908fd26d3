// C ABI of the Fourier neural operator used as the ground-state warm start
// (include/spgpe.h, spgpe_fno_*): parameters, twiddle matrices, and the
// forward pass, gradient and Adam step as sequences of the kernels in
// fno_kernels.cu.  Layout of activations: [batch][channel][n][n], x fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <string>
#include <vector>

#include "fno_internal.h"
#include "spgpe.h"

using namespace spgpe::fno;

namespace {

const double kTwoPi = 6.28318530717958647692528676655900577;

struct Buf {
  float *p = nullptr;
  size_t n = 0;
};

}  // namespace

struct spgpe_fno {
  int cin, cout, W, M, L, H;
  cudaStream_t st = nullptr;
  // flat parameter vector: offsets of P, p, (W_l, w_l, R_l) per layer, Q1, q1, Q2, q2
  long oP, op, oQ1, oq1, oQ2, oq2, nparam = 0;
  std::vector<long> oW, ow, oR;
  float *w = nullptr, *wr = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  void *wb = nullptr;  // bfloat16 weights used in the products
  int t = 0;
  // twiddle matrices for grid size tw_n
  int tw_n = 0;
  float *Exr = nullptr, *Exi = nullptr;
  float2 *Ey = nullptr;
  // workspace for (ws_b, ws_n)
  int ws_b = 0, ws_n = 0;
  std::vector<float *> vs, us;
  std::vector<float2 *> vh;
  float *X1 = nullptr, *hp = nullptr, *h = nullptr, *dh = nullptr, *dv = nullptr, *dv2 = nullptr, *dout = nullptr;
  float2 *oh = nullptr, *G = nullptr, *doh = nullptr;
  float *part = nullptr;
  size_t part_n = 0;
  double *sums = nullptr;
  int *d_flags = nullptr;  // device error flags (a tensor-core wait that ran out)
  double *bscr = nullptr;  // bias-gradient partial sums (64 per channel)
  bool tensor_cores = true;  // SPGPE_FNO_TC=0 keeps every product on the CUDA cores
  std::vector<void *> allocs;
  std::string err;
};

namespace {

int ffail(spgpe_fno *f, int code, const std::string &msg) {
  if (f) f->err = msg;
  return code;
}

#define FCK(f, expr)                                                                          \
  do {                                                                                        \
    cudaError_t _e = (expr);                                                                  \
    if (_e != cudaSuccess) return ffail(f, SPGPE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

template <class T> int falloc(spgpe_fno *f, T **p, size_t count) {
  void *q = nullptr;
  const cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ffail(f, e == cudaErrorMemoryAllocation ? SPGPE_ENOMEM : SPGPE_ECUDA, "cudaMalloc failed");
  }
  f->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return SPGPE_OK;
}

void release(spgpe_fno *f, void *p) {
  for (auto &q : f->allocs)
    if (q == p) {
      cudaFree(q);
      q = nullptr;
    }
}

// Twiddle matrices of the truncated transforms on an n x n grid (FP64, rounded once):
// Exr[x][2k], Exr[x][2k+1] = cos, -sin(2 pi k x / n), k < M (forward along x);
// Ey[j][y] = exp(-2 pi i ky_j y / n), ky_j = j (j < M) or n - 2M + j (forward along y);
// Exi[2k][x], Exi[2k+1][x] = g_k cos, -g_k sin(2 pi k x / n) / n^2 (real part of
// the inverse along x, g_0 = 1, g_k = 2).
int ensure_twiddles(spgpe_fno *f, int n) {
  if (f->tw_n == n) return SPGPE_OK;
  const int M = f->M;
  for (void *p : {(void *)f->Exr, (void *)f->Exi, (void *)f->Ey}) release(f, p);
  f->tw_n = 0;
  std::vector<float> exr((size_t)n * 2 * M), exi((size_t)2 * M * n), ey((size_t)2 * M * n * 2);
  for (int x = 0; x < n; ++x)
    for (int k = 0; k < M; ++k) {
      const double th = kTwoPi * (double)((long)k * x % n) / n, gk = k == 0 ? 1.0 : 2.0;
      exr[(size_t)x * 2 * M + 2 * k] = (float)std::cos(th);
      exr[(size_t)x * 2 * M + 2 * k + 1] = (float)-std::sin(th);
      exi[(size_t)(2 * k) * n + x] = (float)(gk * std::cos(th) / ((double)n * n));
      exi[(size_t)(2 * k + 1) * n + x] = (float)(-gk * std::sin(th) / ((double)n * n));
    }
  for (int j = 0; j < 2 * M; ++j) {
    const long ky = j < M ? j : n - 2 * M + j;
    for (int y = 0; y < n; ++y) {
      const double th = kTwoPi * (double)(ky * y % n) / n;
      ey[((size_t)j * n + y) * 2] = (float)std::cos(th);
      ey[((size_t)j * n + y) * 2 + 1] = (float)-std::sin(th);
    }
  }
  int r;
  if ((r = falloc(f, &f->Exr, exr.size())) || (r = falloc(f, &f->Exi, exi.size())) ||
      (r = falloc(f, &f->Ey, (size_t)2 * M * n)))
    return r;
  FCK(f, cudaMemcpy(f->Exr, exr.data(), exr.size() * sizeof(float), cudaMemcpyHostToDevice));
  FCK(f, cudaMemcpy(f->Exi, exi.data(), exi.size() * sizeof(float), cudaMemcpyHostToDevice));
  FCK(f, cudaMemcpy(f->Ey, ey.data(), ey.size() * sizeof(float), cudaMemcpyHostToDevice));
  f->tw_n = n;
  return SPGPE_OK;
}

int ensure_workspace(spgpe_fno *f, int B, int n) {
  if (f->ws_b >= B && f->ws_n == n) return SPGPE_OK;
  for (float *p : f->vs) release(f, p);
  for (float *p : f->us) release(f, p);
  for (float2 *p : f->vh) release(f, p);
  for (void *p : {(void *)f->X1, (void *)f->hp, (void *)f->h, (void *)f->dh, (void *)f->dv, (void *)f->dv2,
                  (void *)f->dout, (void *)f->oh, (void *)f->G, (void *)f->doh, (void *)f->part, (void *)f->sums})
    release(f, p);
  f->vs.assign(f->L + 1, nullptr);
  f->us.assign(f->L, nullptr);
  f->vh.assign(f->L, nullptr);
  f->ws_b = f->ws_n = 0;
  const size_t P = (size_t)n * n, act = (size_t)B * f->W * P, hid = (size_t)B * f->H * P;
  const size_t spec = (size_t)B * f->W * 2 * f->M * f->M, rows = (size_t)B * f->W * n * f->M;
  int r;
  for (int l = 0; l <= f->L; ++l)
    if ((r = falloc(f, &f->vs[l], act))) return r;
  for (int l = 0; l < f->L; ++l)
    if ((r = falloc(f, &f->us[l], act)) || (r = falloc(f, &f->vh[l], spec))) return r;
  // split-K partials of the weight gradients: batch x splits x (largest weight)
  const int splits = (int)std::max<size_t>(1, P / 1024);
  size_t wmax = std::max<size_t>((size_t)f->W * f->cin, (size_t)f->W * f->W);
  wmax = std::max(wmax, std::max((size_t)f->H * f->W, (size_t)f->cout * f->H));
  f->part_n = (size_t)B * splits * wmax;
  if ((r = falloc(f, &f->X1, rows * 2)) || (r = falloc(f, &f->hp, hid)) || (r = falloc(f, &f->h, hid)) ||
      (r = falloc(f, &f->dh, hid)) || (r = falloc(f, &f->dv, act)) || (r = falloc(f, &f->dv2, act)) ||
      (r = falloc(f, &f->dout, (size_t)B * f->cout * P)) || (r = falloc(f, &f->oh, spec)) ||
      (r = falloc(f, &f->G, rows)) || (r = falloc(f, &f->doh, spec)) || (r = falloc(f, &f->part, f->part_n)) ||
      (r = falloc(f, &f->sums, (size_t)130 * B)))
    return r;
  f->ws_b = B;
  f->ws_n = n;
  return SPGPE_OK;
}

// real GEMM shorthands
GemmR rg(int M, int N, int K, const void *A, bool bf, long sAm, long sAk, const float *Bm, long sBk, long sBn,
         float *C, long sCm, long sCn) {
  GemmR g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = A;
  g.a_bf16 = bf;
  g.sAm = sAm;
  g.sAk = sAk;
  g.B = Bm;
  g.sBk = sBk;
  g.sBn = sBn;
  g.C = C;
  g.sCm = sCm;
  g.sCn = sCn;
  return g;
}

GemmC cg(int M, int N, int K, int batch, const void *A, bool bf, bool ca, long sAm, long sAk, long sAb,
         const float2 *Bm, bool cb, long sBk, long sBn, long sBb, float2 *C, long sCm, long sCn, long sCb,
         float beta = 0.f) {
  GemmC g;
  g.M = M;
  g.N = N;
  g.K = K;
  g.batch = batch;
  g.A = A;
  g.a_bf16 = bf;
  g.conj_a = ca;
  g.conj_b = cb;
  g.sAm = sAm;
  g.sAk = sAk;
  g.sAb = sAb;
  g.B = Bm;
  g.sBk = sBk;
  g.sBn = sBn;
  g.sBb = sBb;
  g.C = C;
  g.sCm = sCm;
  g.sCn = sCn;
  g.sCb = sCb;
  g.beta = beta;
  return g;
}

const void *bfp(const spgpe_fno *f, long off) { return static_cast<const uint16_t *>(f->wb) + off; }

// A real product of the model: the tensor-core path where it applies.
cudaError_t greal(const spgpe_fno *f, GemmR g, cudaStream_t st) {
  g.flags = f->tensor_cores ? f->d_flags : nullptr;
  return gemm_real(g, st);
}

// Report (and clear) an error recorded on the device; after a synchronisation.
int read_flags(spgpe_fno *f) {
  int h = 0;
  FCK(f, cudaMemcpy(&h, f->d_flags, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    FCK(f, cudaMemset(f->d_flags, 0, sizeof(int)));
    return ffail(f, SPGPE_ETIMEOUT, "a tensor-core wait ran out");
  }
  return SPGPE_OK;
}

// grad[M][N] += sum_b sum_p A[b](m, p) Bm[b](p, n): split-K over the points,
// partials reduced in a fixed order.
int wgrad(spgpe_fno *f, int M, int N, long P, int B, const float *A, long sAb, const float *Bm, long sBn, long sBb,
          float *grad) {
  const int splits = (int)std::max<long>(1, P / 1024);
  GemmR g = rg(M, N, (int)P, A, false, P, 1, Bm, 1, sBn, f->part, N, 1);
  g.batch = B;
  g.sAb = sAb;
  g.sBb = sBb;
  g.splits = splits;
  g.partial = true;
  g.sCs = (long)M * N;
  FCK(f, greal(f, g, f->st));
  FCK(f, sum_splits(f->part, (long)M * N, B * splits, grad, true, f->st));
  return SPGPE_OK;
}

int forward(spgpe_fno *f, const float *a, int B, int n, float *out) {
  int r;
  if ((r = ensure_twiddles(f, n)) || (r = ensure_workspace(f, B, n))) return r;
  const long P = (long)n * n, W = f->W, M = f->M, H = f->H;
  const long WP = W * P, SP = 2 * M * M;
  cudaStream_t st = f->st;
  // lift: v0 = P a + p
  GemmR g = rg(W, P, f->cin, bfp(f, f->oP), true, f->cin, 1, a, P, 1, f->vs[0], P, 1);
  g.batch = B;
  g.sBb = (long)f->cin * P;
  g.sCb = WP;
  g.bias = f->wr + f->op;
  FCK(f, greal(f, g, st));
  for (int l = 0; l < f->L; ++l) {
    float *v = f->vs[l], *u = f->us[l];
    // along x: X1 = v Exr, computed as X1^T = Exr^T v^T (the long side as N)
    FCK(f, greal(f, rg(2 * M, B * W * n, n, f->Exr, false, 1, 2 * M, v, 1, n, f->X1, 1, 2 * M), st));
    const float2 *X1c = reinterpret_cast<const float2 *>(f->X1);
    // along y: vh = Ey X1 per (sample, channel)
    FCK(f, gemm_complex(cg(2 * M, M, n, B * W, f->Ey, false, false, n, 1, 0, X1c, false, M, 1, n * M, f->vh[l], M, 1,
                           SP),
                        st));
    // channel mixing per mode: oh[b][o][m] = sum_c R[m][o][c] vh[b][c][m]
    FCK(f, gemm_complex(cg(W, B, W, SP, bfp(f, f->oR[l]), true, false, W, 1, W * W, f->vh[l], false, SP, W * SP, 1,
                           f->oh, SP, W * SP, 1),
                        st));
    // inverse along y: G = conj(Ey)^T oh per (sample, channel)
    FCK(f, gemm_complex(cg(n, M, 2 * M, B * W, f->Ey, false, true, 1, n, 0, f->oh, false, M, 1, SP, f->G, M, 1, n * M),
                        st));
    // real part of the inverse along x: u = G Exi
    FCK(f, greal(f, rg(B * W * n, n, 2 * M, reinterpret_cast<const float *>(f->G), false, 2 * M, 1, f->Exi, n, 1,
                        u, n, 1),
                     st));
    // u += W_l v + w_l
    g = rg(W, P, W, bfp(f, f->oW[l]), true, W, 1, v, P, 1, u, P, 1);
    g.batch = B;
    g.sBb = WP;
    g.sCb = WP;
    g.beta = 1.f;
    g.bias = f->wr + f->ow[l];
    FCK(f, greal(f, g, st));
    if (l < f->L - 1) {
      FCK(f, gelu_forward(u, f->vs[l + 1], (long)B * WP, st));
    } else {
      FCK(f, cudaMemcpyAsync(f->vs[l + 1], u, (size_t)B * WP * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
  }
  // projection
  g = rg(H, P, W, bfp(f, f->oQ1), true, W, 1, f->vs[f->L], P, 1, f->hp, P, 1);
  g.batch = B;
  g.sBb = WP;
  g.sCb = H * P;
  g.bias = f->wr + f->oq1;
  FCK(f, greal(f, g, st));
  FCK(f, gelu_forward(f->hp, f->h, (long)B * H * P, st));
  g = rg(f->cout, P, H, bfp(f, f->oQ2), true, H, 1, f->h, P, 1, out, P, 1);
  g.batch = B;
  g.sBb = H * P;
  g.sCb = (long)f->cout * P;
  g.bias = f->wr + f->oq2;
  FCK(f, greal(f, g, st));
  return SPGPE_OK;
}

// Loss (mean relative squared error) and gradient of all parameters into f->g.
int gradient(spgpe_fno *f, const float *a, const float *target, int B, int n, float *out, double *loss) {
  int r = forward(f, a, B, n, out);
  if (r) return r;
  const long P = (long)n * n, W = f->W, M = f->M, H = f->H, C = f->cout;
  const long WP = W * P, SP = 2 * M * M;
  cudaStream_t st = f->st;
  FCK(f, cudaMemsetAsync(f->g, 0, (size_t)f->nparam * sizeof(float), st));
  FCK(f, loss_terms(out, target, C * P, B, f->sums, f->dout, st));
  // output layer
  if ((r = wgrad(f, C, H, P, B, f->dout, C * P, f->h, P, H * P, f->g + f->oQ2))) return r;
  FCK(f, bias_gradient(f->dout, B, C, P, f->g + f->oq2, f->bscr, st));
  GemmR g = rg(H, P, C, bfp(f, f->oQ2), true, 1, H, f->dout, P, 1, f->dh, P, 1);
  g.batch = B;
  g.sBb = C * P;
  g.sCb = H * P;
  FCK(f, greal(f, g, st));
  FCK(f, gelu_backward(f->hp, f->dh, (long)B * H * P, st));
  if ((r = wgrad(f, H, W, P, B, f->dh, H * P, f->vs[f->L], P, WP, f->g + f->oQ1))) return r;
  FCK(f, bias_gradient(f->dh, B, H, P, f->g + f->oq1, f->bscr, st));
  g = rg(W, P, H, bfp(f, f->oQ1), true, 1, W, f->dh, P, 1, f->dv, P, 1);
  g.batch = B;
  g.sBb = H * P;
  g.sCb = WP;
  FCK(f, greal(f, g, st));
  float *du = f->dv, *dvn = f->dv2;
  for (int l = f->L - 1; l >= 0; --l) {
    if (l < f->L - 1) FCK(f, gelu_backward(f->us[l], du, (long)B * WP, st));
    if ((r = wgrad(f, W, W, P, B, du, WP, f->vs[l], P, WP, f->g + f->oW[l]))) return r;
    FCK(f, bias_gradient(du, B, W, P, f->g + f->ow[l], f->bscr, st));
    // dv = W_l^T du
    g = rg(W, P, W, bfp(f, f->oW[l]), true, 1, W, du, P, 1, dvn, P, 1);
    g.batch = B;
    g.sBb = WP;
    g.sCb = WP;
    FCK(f, greal(f, g, st));
    // spectral part: dG = du Exi^T (into X1; as dG^T = Exi du^T), doh = Ey dG
    FCK(f, greal(f, rg(2 * M, B * W * n, n, f->Exi, false, n, 1, du, 1, n, f->X1, 1, 2 * M), st));
    const float2 *dG = reinterpret_cast<const float2 *>(f->X1);
    FCK(f, gemm_complex(cg(2 * M, M, n, B * W, f->Ey, false, false, n, 1, 0, dG, false, M, 1, n * M, f->doh, M, 1, SP),
                        st));
    // dR[m] += sum_b doh[b][:, m] vh[b][:, m]^H
    FCK(f, gemm_complex(cg(W, W, B, SP, f->doh, false, false, SP, W * SP, 1, f->vh[l], true, W * SP, SP, 1,
                           reinterpret_cast<float2 *>(f->g + f->oR[l]), W, 1, W * W, 1.f),
                        st));
    // dvh[b][c][m] = sum_o conj(R[m][o][c]) doh[b][o][m]  (into oh)
    FCK(f, gemm_complex(cg(W, B, W, SP, bfp(f, f->oR[l]), true, true, 1, W, W * W, f->doh, false, SP, W * SP, 1,
                           f->oh, SP, W * SP, 1),
                        st));
    // dX1 = conj(Ey)^T dvh (into G), dv += dX1 Exr^T
    FCK(f, gemm_complex(cg(n, M, 2 * M, B * W, f->Ey, false, true, 1, n, 0, f->oh, false, M, 1, SP, f->G, M, 1, n * M),
                        st));
    g = rg(B * W * n, n, 2 * M, reinterpret_cast<const float *>(f->G), false, 2 * M, 1, f->Exr, 1, 2 * M, dvn, n, 1);
    g.beta = 1.f;
    FCK(f, greal(f, g, st));
    std::swap(du, dvn);
  }
  if ((r = wgrad(f, W, f->cin, P, B, du, WP, a, P, (long)f->cin * P, f->g + f->oP))) return r;
  FCK(f, bias_gradient(du, B, W, P, f->g + f->op, f->bscr, st));
  if (loss) {
    std::vector<double> s((size_t)2 * B);
    FCK(f, cudaMemcpyAsync(s.data(), f->sums, s.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    FCK(f, cudaStreamSynchronize(st));
    if ((r = read_flags(f))) return r;
    double l = 0.0;
    for (int b = 0; b < B; ++b) l += s[2 * (size_t)b] / s[2 * (size_t)b + 1];
    *loss = l / B;
  }
  return SPGPE_OK;
}

// Seeded initial weights (SplitMix64 uniforms): matrices U(-1/sqrt(fan_in),
// 1/sqrt(fan_in)), biases zero, spectral weights U(0, 1) / (W W) in both parts.
void init_params(const spgpe_fno *f, unsigned long long seed, std::vector<float> &h) {
  h.assign((size_t)f->nparam, 0.f);
  unsigned long long c = 0;
  auto u01 = [&]() {
    unsigned long long z = seed + (++c) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
  };
  auto mat = [&](long off, long rows, long cols) {
    const double b = 1.0 / std::sqrt((double)cols);
    for (long i = 0; i < rows * cols; ++i) h[(size_t)(off + i)] = (float)(b * (2.0 * u01() - 1.0));
  };
  mat(f->oP, f->W, f->cin);
  for (int l = 0; l < f->L; ++l) {
    mat(f->oW[l], f->W, f->W);
    const long nr = 2L * f->M * f->M * f->W * f->W * 2;
    for (long i = 0; i < nr; ++i) h[(size_t)(f->oR[l] + i)] = (float)(u01() / ((double)f->W * f->W));
  }
  mat(f->oQ1, f->H, f->W);
  mat(f->oQ2, f->cout, f->H);
}

int check_shape(spgpe_fno *f, const void *a, int B, int n) {
  if (!f || !a || B < 1 || n < 2 * f->M || n > 4096 || (n & (n - 1)))
    return ffail(f, SPGPE_EINVAL, "bad input, batch or grid size (n a power of two, n >= 2 * modes)");
  return SPGPE_OK;
}

}  // namespace

extern "C" {

int spgpe_fno_create(spgpe_fno **out, int cin, int cout, int width, int modes, int layers, int hidden,
                     unsigned long long seed, void *cuda_stream) {
  if (!out) return SPGPE_EINVAL;
  *out = nullptr;
  if (cin < 1 || cout < 1 || width < 1 || modes < 1 || layers < 1 || hidden < 1 || width > 1024 || hidden > 4096 ||
      cin > 1024 || cout > 1024 || modes > 1024 || layers > 64)
    return SPGPE_EINVAL;
  spgpe_fno *f = new (std::nothrow) spgpe_fno();
  if (!f) return SPGPE_ENOMEM;
  f->cin = cin;
  f->cout = cout;
  f->W = width;
  f->M = modes;
  f->L = layers;
  f->H = hidden;
  f->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  long o = 0;
  f->oP = o;
  o += (long)width * cin;
  f->op = o;
  o += width;
  for (int l = 0; l < layers; ++l) {
    f->oW.push_back(o);
    o += (long)width * width;
    f->ow.push_back(o);
    o += width;
    f->oR.push_back(o);
    o += 2L * modes * modes * width * width * 2;
  }
  f->oQ1 = o;
  o += (long)hidden * width;
  f->oq1 = o;
  o += hidden;
  f->oQ2 = o;
  o += (long)cout * hidden;
  f->oq2 = o;
  o += cout;
  f->nparam = o;
  int r;
  const size_t np = (size_t)o;
  if ((r = falloc(f, &f->w, np)) || (r = falloc(f, &f->wr, np)) || (r = falloc(f, &f->g, np)) ||
      (r = falloc(f, &f->m, np)) || (r = falloc(f, &f->v, np)) || (r = falloc(f, (uint16_t **)&f->wb, np)) ||
      (r = falloc(f, &f->d_flags, 1)) ||
      (r = falloc(f, &f->bscr, (size_t)64 * std::max(std::max(width, hidden), std::max(cin, cout))))) {
    spgpe_fno_destroy(f);
    return r;
  }
  if (cudaMemset(f->d_flags, 0, sizeof(int)) != cudaSuccess) {
    spgpe_fno_destroy(f);
    return SPGPE_ECUDA;
  }
  const char *tc = std::getenv("SPGPE_FNO_TC");
  f->tensor_cores = !(tc && tc[0] == '0');
  std::vector<float> h;
  init_params(f, seed, h);
  if (spgpe_fno_set_params(f, h.data()) != SPGPE_OK) {
    spgpe_fno_destroy(f);
    return SPGPE_ECUDA;
  }
  *out = f;
  return SPGPE_OK;
}

long spgpe_fno_num_params(const spgpe_fno *f) { return f ? f->nparam : 0; }

const char *spgpe_fno_last_error(const spgpe_fno *f) { return f ? f->err.c_str() : "NULL model"; }

int spgpe_fno_get_params(spgpe_fno *f, float *host) {
  if (!f || !host) return ffail(f, SPGPE_EINVAL, "NULL argument");
  FCK(f, cudaMemcpyAsync(host, f->w, (size_t)f->nparam * sizeof(float), cudaMemcpyDeviceToHost, f->st));
  FCK(f, cudaStreamSynchronize(f->st));
  return SPGPE_OK;
}

int spgpe_fno_set_params(spgpe_fno *f, const float *host) {
  if (!f || !host) return ffail(f, SPGPE_EINVAL, "NULL argument");
  const size_t bytes = (size_t)f->nparam * sizeof(float);
  FCK(f, cudaMemcpyAsync(f->w, host, bytes, cudaMemcpyHostToDevice, f->st));
  FCK(f, round_weights(f->w, f->wb, f->wr, f->nparam, f->st));
  FCK(f, cudaMemsetAsync(f->m, 0, bytes, f->st));
  FCK(f, cudaMemsetAsync(f->v, 0, bytes, f->st));
  FCK(f, cudaStreamSynchronize(f->st));
  f->t = 0;
  return SPGPE_OK;
}

int spgpe_fno_forward(spgpe_fno *f, const float *a, int batch, int n, float *out) {
  int r = check_shape(f, a, batch, n);
  if (r) return r;
  if (!out) return ffail(f, SPGPE_EINVAL, "NULL output");
  return forward(f, a, batch, n, out);
}

int spgpe_fno_gradient(spgpe_fno *f, const float *a, const float *target, int batch, int n, float *out,
                       double *loss, float *grad_host) {
  int r = check_shape(f, a, batch, n);
  if (r) return r;
  if (!target || !out) return ffail(f, SPGPE_EINVAL, "NULL target or output");
  if ((r = gradient(f, a, target, batch, n, out, loss))) return r;
  if (grad_host) {
    FCK(f, cudaMemcpyAsync(grad_host, f->g, (size_t)f->nparam * sizeof(float), cudaMemcpyDeviceToHost, f->st));
    FCK(f, cudaStreamSynchronize(f->st));
    if ((r = read_flags(f))) return r;
  }
  return SPGPE_OK;
}

int spgpe_fno_train_step(spgpe_fno *f, const float *a, const float *target, int batch, int n, float *out,
                         double lr, double *loss) {
  int r = check_shape(f, a, batch, n);
  if (r) return r;
  if (!target || !out || !(lr > 0) || !std::isfinite(lr)) return ffail(f, SPGPE_EINVAL, "bad target, output or lr");
  if ((r = gradient(f, a, target, batch, n, out, loss))) return r;
  ++f->t;
  FCK(f, adam_update(f->w, f->wb, f->wr, f->g, f->m, f->v, f->nparam, (float)lr, f->t, f->st));
  return SPGPE_OK;
}

void spgpe_fno_destroy(spgpe_fno *f) {
  if (!f) return;
  cudaStreamSynchronize(f->st);
  for (void *p : f->allocs)
    if (p) cudaFree(p);
  delete f;
}

}  // extern "C"
