// Tensor-core (tcgen05) products of the Fourier neural operator's pointwise
// channel maps: C[b](m, p) = sum_k A(m, k) X[b](k, p) (+ beta C + bias[m]),
// with A a bfloat16 weight matrix (any strides; NC = 64 or 128 rows, K = 64
// or 128) and X the float32 activations [k][p] (p contiguous, P a multiple
// of 128).
//
// The product runs transposed on the tensor cores: each tile is 128 points
// (the MMA's M), NC channels (its N) and K input channels, accumulated in
// tensor memory (TMEM, one 32-bit column per output channel, one lane per
// point).  The weights are exact in bfloat16; each float32 activation x is
// split into three bfloat16 terms, x = h + m + l up to the last bit of its
// 24-bit significand (h = bf16(x), m = bf16(x - h), l = bf16(x - h - m)),
// so that A X = A h + A m + A l with every product exact and float32
// accumulation: three MMA passes per K step instead of one, at float32
// accuracy (the technique of splitting a float32 operand into bfloat16
// terms: Henry, Tang and Heinecke, "Leveraging the bfloat16 artificial
// intelligence datatype for higher-precision computations", ARITH 2019).
//
// Shared-memory operands are K-major with the 128-byte swizzle (rows of 64
// bfloat16, 16-byte chunk c of row r stored at chunk c ^ (r & 7), 1024-byte
// aligned blocks of 8 rows), written by the threads from registers (the
// activations need the split, so no TMA here); one thread issues the MMAs
// and commits them to an mbarrier that every thread waits on (bounded).
// Persistent CTAs of 128 threads loop over tiles; the weights are staged once.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "async_copy.cuh"
#include "fno_internal.h"

namespace spgpe {
namespace fno {

namespace {

constexpr int kTcRows = 128;              // points per tile (MMA M)
constexpr int kKBlock = 64;               // bfloat16 per 128-byte swizzled row
constexpr int kRowBytes = 128;

__device__ __forceinline__ uint32_t sw128(int row, int chunk) {
  return (uint32_t)row * kRowBytes + ((uint32_t)(chunk ^ (row & 7)) << 4);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(const void *base) {
  const uint64_t a = smem_addr(base);
  return ((a >> 4) & 0x3FFFull) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16: float32 accumulator, bfloat16 A and
// B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D (TMEM) [+]= A (smem) x B (smem)
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on the mbarrier once every MMA this thread issued has completed.
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Shared memory: three activation terms [term][kb][128 rows][128 B], the
// weights [kb][NC rows][128 B], the mbarrier and the TMEM address slot.
template <int NC, int KB> struct TcSmem {
  static constexpr size_t kTerm = (size_t)KB * kTcRows * kRowBytes;
  static constexpr size_t kA = 3 * kTerm;
  static constexpr size_t kB = (size_t)KB * NC * kRowBytes;
  static constexpr size_t kBytes = 1024 /* alignment slack */ + kA + kB + 16;
};

template <int NC, int KB>
__global__ void __launch_bounds__(128) gemm_tc(int ntiles, int tiles_per_batch, const __nv_bfloat16 *__restrict__ A,
                                               long sAm, long sAk, const float *__restrict__ X, long sXk, long sXb,
                                               float *C, long sCm, long sCb, float beta,
                                               const float *__restrict__ bias, int *flags) {
  constexpr int K = KB * kKBlock;
  using S = TcSmem<NC, KB>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *sA = sm;            // activation terms
  unsigned char *sB = sm + S::kA;    // weights
  uint64_t *bar = reinterpret_cast<uint64_t *>(sB + S::kB);
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tmem_alloc(slot, NC);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  // weights, once: row m (output channel), chunk j holds k = 8 j .. 8 j + 7
  for (int e = tid; e < NC * (K / 8); e += blockDim.x) {
    const int m = e / (K / 8), j = e - m * (K / 8);
    const int kb = j / 8, jc = j % 8;
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long k0 = 8L * j + 2 * i;
      w[i] = pack_bf16(A[m * sAm + k0 * sAk], A[m * sAm + (k0 + 1) * sAk]);
    }
    *reinterpret_cast<uint4 *>(sB + (size_t)kb * NC * kRowBytes + sw128(m, jc)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  constexpr uint32_t idesc = idesc_bf16(kTcRows, NC);
  // Software pipeline: while the tensor cores and the epilogue work on one
  // tile, this thread's activations of the next tile (and, for 64 output
  // channels, the previous C values of the current one) are already in flight.
  float xr[K];
  auto load_x = [&](int tile) {
    const int b = tile / tiles_per_batch;
    const float *xs = X + b * sXb + (long)(tile - b * tiles_per_batch) * kTcRows + tid;
#pragma unroll
    for (int k = 0; k < K; ++k) xr[k] = xs[(long)k * sXk];
  };
  constexpr bool kPreC = NC == 64;
  float cpre[kPreC ? NC : 1];
  bool ok = true;
  int it = 0;
  int tile = blockIdx.x;
  if (tile < ntiles) load_x(tile);
  for (; tile < ntiles && ok; tile += gridDim.x, ++it) {
    const int b = tile / tiles_per_batch;
    const long p0 = (long)(tile - b * tiles_per_batch) * kTcRows;
    // this thread's point p0 + tid: three bfloat16 terms per activation
#pragma unroll
    for (int j = 0; j < K / 8; ++j) {
      uint32_t hw[4], mw[4], lw[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        __nv_bfloat16 h[2], md[2], lo[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float v = xr[8 * j + 2 * i + q];
          h[q] = __float2bfloat16_rn(v);
          const float r1 = v - __bfloat162float(h[q]);
          md[q] = __float2bfloat16_rn(r1);
          lo[q] = __float2bfloat16_rn(r1 - __bfloat162float(md[q]));
        }
        hw[i] = pack_bf16(h[0], h[1]);
        mw[i] = pack_bf16(md[0], md[1]);
        lw[i] = pack_bf16(lo[0], lo[1]);
      }
      const size_t off = (size_t)(j / 8) * kTcRows * kRowBytes + sw128(tid, j % 8);
      *reinterpret_cast<uint4 *>(sA + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4 *>(sA + S::kTerm + off) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
      *reinterpret_cast<uint4 *>(sA + 2 * S::kTerm + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    // the tensor cores read shared memory through the async proxy
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll 1
      for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          const uint64_t ad = sw128_desc(sA + t * S::kTerm + (size_t)kb * kTcRows * kRowBytes);
          const uint64_t bd = sw128_desc(sB + (size_t)kb * NC * kRowBytes);
#pragma unroll
          for (int kk = 0; kk < kKBlock / 16; ++kk)  // 16 bfloat16 = 32 bytes per MMA
            umma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (t | kb | kk) != 0);
        }
      umma_commit(bar);
    }
    // lane (warp, lane) holds point p0 + 32 warp + lane, one TMEM column per channel
    const long p = p0 + 32 * warp + lane;
    float *cb = C + b * sCb + p;
    if (tile + (int)gridDim.x < ntiles) load_x(tile + gridDim.x);
    if constexpr (kPreC) {
      if (beta != 0.f)
#pragma unroll
        for (int m = 0; m < NC; ++m) cpre[m] = cb[m * sCm];
    }
    ok = mbar_wait_bounded(bar, (uint32_t)(it & 1));
    if (!__syncthreads_and(ok)) {
      // the MMAs never completed: record it, give them one more bounded wait
      if (tid == 0) atomicOr(flags, kErrTimeout);
      mbar_wait_bounded(bar, (uint32_t)(it & 1));
      ok = false;
      break;
    }
    tc_fence_after();
#pragma unroll
    for (int c0 = 0; c0 < NC; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int m = c0 + i;
        float o = v[i];
        if (beta != 0.f) {
          if constexpr (kPreC) o = fmaf(beta, cpre[m], o);
          else o = fmaf(beta, cb[m * sCm], o);
        }
        if (bias) o += bias[m];
        cb[m * sCm] = o;
      }
    }
    // every lane is read before the next tile's MMAs overwrite the accumulator
    tc_fence_before();
    __syncthreads();
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, NC);
  }
}

template <int NC, int KB>
cudaError_t launch_tc(const GemmR &g, cudaStream_t st) {
  auto kern = gemm_tc<NC, KB>;
  const size_t smem = TcSmem<NC, KB>::kBytes;
  static int granted = 0, occ = 0, sms = 0;
  if (!granted) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    granted = 1;
  }
  const int tpb = g.N / kTcRows, ntiles = tpb * g.batch;
  const int grid = std::max(1, std::min(ntiles, std::max(1, occ) * sms));
  kern<<<grid, 128, smem, st>>>(ntiles, tpb, static_cast<const __nv_bfloat16 *>(g.A), g.sAm, g.sAk, g.B, g.sBk,
                                g.sBb, g.C, g.sCm, g.sCb, g.beta, g.bias, g.flags);
  return cudaGetLastError();
}

// Weight gradients on the tensor cores: part[b splits + s](m, n) =
// sum over points p of split s of X[b](m, p) Y[b](n, p), m < M, n < N, both
// operands float32 with unit stride along p (the K dimension of the MMA).  Each
// operand is split into two bfloat16 terms (x = h + l, 16 significant bits),
// and the three products h h', h l', l h' are accumulated (the dropped l l' is
// below 2^-16 of the result).  The MMA tile is 128 rows of X (M <= MR = 64 or
// 128; the rows from M on stay zero) by NC = 16, 64 or 128 rows of Y (N <= NC,
// likewise).  One CTA per (sample, split), its 64-point blocks streamed
// through registers one block ahead of the MMAs.
template <int MR, int NC> struct WgSmem {
  static constexpr size_t kA = (size_t)kTcRows * kRowBytes;  // one term of X
  static constexpr size_t kB = (size_t)NC * kRowBytes;       // one term of Y
  static constexpr size_t kBytes = 1024 + 2 * kA + 2 * kB + 16;
};

template <int MR, int NC>
__global__ void __launch_bounds__(128) gemm_tc_wgrad(int M, int N, int splits, int ks, const float *__restrict__ X,
                                                     long sXm, long sXb, const float *__restrict__ Y, long sYn,
                                                     long sYb, float *part, long sPs, int *flags) {
  using S = WgSmem<MR, NC>;
  constexpr uint32_t kCols = NC < 32 ? 32 : NC;  // TMEM allocations are powers of two from 32 columns
  constexpr int CH = (MR + NC) * 8 / 128;  // 16-byte chunks of one 64-point block per thread
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *sA = sm, *sB = sm + 2 * S::kA;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sB + 2 * S::kB);
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x / splits, sp = blockIdx.x - b * splits;
  const long k0 = (long)sp * ks;
  const float *xb = X + b * sXb + k0, *yb = Y + b * sYb + k0;

  if (warp == 0) {
    tmem_alloc(slot, kCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  // rows M..127 of both X terms and N..NC-1 of both Y terms stay zero
  for (int e = tid; e < (kTcRows - M) * 8; e += blockDim.x) {
    const int r = M + e / 8, c = e % 8;
    *reinterpret_cast<uint4 *>(sA + sw128(r, c)) = make_uint4(0, 0, 0, 0);
    *reinterpret_cast<uint4 *>(sA + S::kA + sw128(r, c)) = make_uint4(0, 0, 0, 0);
  }
  for (int e = tid; e < (NC - N) * 8; e += blockDim.x) {
    const int r = N + e / 8, c = e % 8;
    *reinterpret_cast<uint4 *>(sB + sw128(r, c)) = make_uint4(0, 0, 0, 0);
    *reinterpret_cast<uint4 *>(sB + S::kB + sw128(r, c)) = make_uint4(0, 0, 0, 0);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  constexpr uint32_t idesc = idesc_bf16(kTcRows, NC);
  // chunk q of a block: rows 0..MR-1 of X then rows of Y, 8 chunks (64 points) per row
  float4 xr[CH][2];
  // valid rows only (the others keep their zeros)
  auto valid = [&](int r) { return r < MR ? r < M : r - MR < N; };
  auto load = [&](long kk) {
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int e = tid + q * 128, r = e / 8, c = e % 8;
      if (valid(r)) {
        const float *src = r < MR ? xb + r * sXm + kk + 8 * c : yb + (r - MR) * sYn + kk + 8 * c;
        xr[q][0] = *reinterpret_cast<const float4 *>(src);
        xr[q][1] = *reinterpret_cast<const float4 *>(src + 4);
      }
    }
  };
  auto split2 = [&](float v, __nv_bfloat16 &h, __nv_bfloat16 &l) {
    h = __float2bfloat16_rn(v);
    l = __float2bfloat16_rn(v - __bfloat162float(h));
  };
  bool ok = true;
  const int nblk = ks / kKBlock;
  load(0);
  for (int blk = 0; blk < nblk && ok; ++blk) {
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int e = tid + q * 128, r = e / 8, c = e % 8;
      if (!valid(r)) continue;
      const float v[8] = {xr[q][0].x, xr[q][0].y, xr[q][0].z, xr[q][0].w,
                          xr[q][1].x, xr[q][1].y, xr[q][1].z, xr[q][1].w};
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        __nv_bfloat16 h0, l0, h1, l1;
        split2(v[2 * i], h0, l0);
        split2(v[2 * i + 1], h1, l1);
        hw[i] = pack_bf16(h0, h1);
        lw[i] = pack_bf16(l0, l1);
      }
      unsigned char *dst = r < MR ? sA + sw128(r, c) : sB + sw128(r - MR, c);
      const size_t term = r < MR ? S::kA : S::kB;
      *reinterpret_cast<uint4 *>(dst) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4 *>(dst + term) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint64_t ah = sw128_desc(sA), al = sw128_desc(sA + S::kA);
      const uint64_t bh = sw128_desc(sB), bl = sw128_desc(sB + S::kB);
#pragma unroll
      for (int kk = 0; kk < kKBlock / 16; ++kk) {
        umma_bf16(tmem, ah + 2 * kk, bh + 2 * kk, idesc, (blk | kk) != 0);
        umma_bf16(tmem, ah + 2 * kk, bl + 2 * kk, idesc, 1);
        umma_bf16(tmem, al + 2 * kk, bh + 2 * kk, idesc, 1);
      }
      umma_commit(bar);
    }
    if (blk + 1 < nblk) load((long)(blk + 1) * kKBlock);
    // the next block's operands go into the same buffers: wait for these MMAs
    ok = mbar_wait_bounded(bar, (uint32_t)(blk & 1));
    if (!__syncthreads_and(ok)) {
      if (tid == 0) atomicOr(flags, kErrTimeout);
      mbar_wait_bounded(bar, (uint32_t)(blk & 1));
      ok = false;
    }
  }
  if (ok) {
    tc_fence_after();
    // rows 0..M-1 of the accumulator, columns 0..N-1: lanes of the first warps
    if (32 * warp < M) {
      const int m = 32 * warp + lane;
      float *out = part + (long)blockIdx.x * sPs + (long)m * N;
#pragma unroll
      for (int c0 = 0; c0 < NC; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
        tmem_ld_wait();
        if (m < M)
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c0 + i < N) out[c0 + i] = v[i];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kCols);
  }
}

template <int MR, int NC>
cudaError_t launch_wgrad(const GemmR &g, cudaStream_t st) {
  auto kern = gemm_tc_wgrad<MR, NC>;
  const size_t smem = WgSmem<MR, NC>::kBytes;
  static int granted = 0;
  if (!granted) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    granted = 1;
  }
  kern<<<g.batch * g.splits, 128, smem, st>>>(g.M, g.N, g.splits, g.K / g.splits, static_cast<const float *>(g.A),
                                              g.sAm, g.sAb, g.B, g.sBn, g.sBb, g.C, g.sCs, g.flags);
  return cudaGetLastError();
}

}  // namespace

namespace {
// split-K weight gradients of two float32 operands with unit stride along K
bool wgrad_applies(const GemmR &g) {
  return !g.a_bf16 && g.flags && g.partial && g.sAk == 1 && g.sBk == 1 && g.sCm == g.N && g.sCn == 1 &&
         g.sCs == (long)g.M * g.N && g.M >= 1 && g.M <= 128 && g.N >= 1 && g.N <= 128 && g.splits >= 1 &&
         g.K % g.splits == 0 && (g.K / g.splits) % kKBlock == 0 && g.sAm % 4 == 0 && g.sBn % 4 == 0 &&
         g.sAb % 4 == 0 && g.sBb % 4 == 0 && (reinterpret_cast<uintptr_t>(g.A) & 15) == 0 &&
         (reinterpret_cast<uintptr_t>(g.B) & 15) == 0 && (reinterpret_cast<uintptr_t>(g.C) & 15) == 0;
}
}  // namespace

bool gemm_tc_applies(const GemmR &g) {
  if (wgrad_applies(g)) return true;
  return g.a_bf16 && g.flags && !g.partial && g.splits == 1 && g.alpha == 1.f && g.sAb == 0 && g.sBn == 1 &&
         g.sCn == 1 && (g.M == 64 || g.M == 128) && (g.K == 64 || g.K == 128) && g.N % kTcRows == 0 &&
         g.N >= kTcRows;
}

cudaError_t gemm_real_tc(const GemmR &g, cudaStream_t st) {
  if (!gemm_tc_applies(g)) return cudaErrorNotSupported;
  if (wgrad_applies(g)) {
    if (g.M <= 64) {
      if (g.N <= 16) return launch_wgrad<64, 16>(g, st);
      return g.N <= 64 ? launch_wgrad<64, 64>(g, st) : launch_wgrad<64, 128>(g, st);
    }
    if (g.N <= 16) return launch_wgrad<128, 16>(g, st);
    return g.N <= 64 ? launch_wgrad<128, 64>(g, st) : launch_wgrad<128, 128>(g, st);
  }
  if (g.M == 64) return g.K == 64 ? launch_tc<64, 1>(g, st) : launch_tc<64, 2>(g, st);
  return g.K == 64 ? launch_tc<128, 1>(g, st) : launch_tc<128, 2>(g, st);
}

}  // namespace fno
}  // namespace spgpe
