// Persistent versions of the row and column passes: each block loops over
// tiles, and the tile after next is already streaming into shared memory
// (double buffering, mbarrier-tracked) while the current one is transformed,
// so HBM latency overlaps the FFT arithmetic instead of stalling it.
//
// Row pass: a tile is `rows` rows of one instance; the two components arrive
// as two contiguous bulk copies (cp.async.bulk), optionally followed by the
// instance's x step table.  Column pass: a tile is C adjacent columns of one
// component, loaded as 2D TMA boxes (cp.async.bulk.tensor) of C columns by up
// to 256 rows.  Results are stored straight from registers.  Every wait is
// bounded; a timeout sets an error bit and the block stops.
#pragma once
#include <cuda.h>

#include "async_copy.cuh"
#include "kernels.cuh"

namespace spgpe {

constexpr int kPipe = 2;  // tile buffers per block

// Shared-memory plan of the persistent column pass.
__host__ __device__ constexpr size_t colp_buf_bytes(int n, int c, int es) {
  return ((size_t)col_smem_elems(n, c, es) * es + 127) / 128 * 128;
}

// A wait for tile i ran out: record the error, then give the other copy this
// block still has in flight (tile + gridDim.x, if it was issued) its own
// bounded wait, so the block does not exit with a transfer landing in its
// shared memory.
__device__ __forceinline__ void drain_after_timeout(uint64_t *bar, int i, int tile, int ntiles, int *flags) {
  if (threadIdx.x == 0) {
    atomicOr(flags, kErrTimeout);
    if (tile + (int)gridDim.x < ntiles) mbar_wait_bounded(&bar[(i + 1) % kPipe], (uint32_t)(((i + 1) / kPipe) & 1));
  }
}

// Shared-memory plan of the persistent row pass (host and device agree).
__host__ __device__ constexpr size_t rowp_buf_bytes(int n, int rows, int es, bool with_tab) {
  // exchange / dense tile region, then the x step table (n q4 = n * 2 * es bytes)
  return (((size_t)rows * row_stride(n, es) * es + (with_tab ? (size_t)n * 2 * es : 0)) + 127) / 128 * 128;
}

template <class T, int LOGN, int LOGE, int F>
__global__ void __launch_bounds__(2 * kRowMaxThreads) row_pass_p(const RowArgs a, int ntiles) {
  constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
  constexpr int ES = sizeof(cx<T>);
  constexpr int PADN = row_pad_n(N, ES), RS = row_stride(N, ES);
  constexpr bool NEEDTAB = (F & (F_REND | F_RSTART)) != 0;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rows = a.rows;
  const bool tab_smem = NEEDTAB && a.tab_in_smem;
  const size_t bufb = rowp_buf_bytes(N, rows, ES, tab_smem);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + kPipe * bufb);
  const RowPlace pl = row_place<TT>();
  const int groups = a.ny / rows;  // tiles per instance
  const uint32_t rowbytes = (uint32_t)rows * N * ES;

  auto buf = [&](int s) { return reinterpret_cast<cx<T> *>(smem_raw + s * bufb); };
  auto issue = [&](int tile, int s) {
    const int inst = tile / groups, y0 = (tile - inst * groups) * rows;
    const cx<T> *src = reinterpret_cast<const cx<T> *>(a.psi) + ((long)inst * 2 * a.ny + y0) * N;
    const uint32_t tabbytes = tab_smem ? (uint32_t)(N * sizeof(q4<T>)) : 0u;
    mbar_expect_tx(&bar[s], 2 * rowbytes + tabbytes);
    bulk_g2s(buf(s), src, rowbytes, &bar[s]);
    bulk_g2s(buf(s) + rows * N, src + (long)a.ny * N, rowbytes, &bar[s]);
    if (tab_smem)
      bulk_g2s(reinterpret_cast<unsigned char *>(buf(s)) + (size_t)rows * RS * ES,
               reinterpret_cast<const q4<T> *>(a.tabx) + (long)inst * N, tabbytes, &bar[s]);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kPipe; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
    for (int s = 0; s < kPipe; ++s)
      if (blockIdx.x + s * gridDim.x < ntiles) issue(blockIdx.x + s * gridDim.x, s);
  }
  __syncthreads();

  int i = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    const int s = i % kPipe;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((i / kPipe) & 1));
    if (!__syncthreads_and(ok)) {
      drain_after_timeout(bar, i, tile, ntiles, a.flags);
      return;
    }
    const int inst = tile / groups, group = tile - inst * groups;
    const int y = group * rows + pl.lrow;
    cx<T> *b = buf(s);
    cx<T> v[1][E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[0][m] = b[(pl.comp * rows + pl.lrow) * N + pl.t + m * TT];
    __syncthreads();  // the dense tile is read; its space now serves the exchanges
    const RowAcc<T, row_warp_local(TT)> acc{b + pl.lrow * RS + pl.comp * PADN, 0, pl.mask};
    const q4<T> *tab = tab_smem ? reinterpret_cast<const q4<T> *>(reinterpret_cast<unsigned char *>(b) +
                                                                  (size_t)rows * RS * ES)
                                : reinterpret_cast<const q4<T> *>(a.tabx) + (long)inst * N;
    double nsum[2] = {0.0, 0.0};
    row_compute<T, LOGN, LOGE, F>(v, pl.t, pl.comp, pl.mask, pl.half, inst, y, acc, tab, a, nsum);
    if constexpr (F & F_PART) row_partials(a, inst, group, groups, nsum);
    cx<T> *p = reinterpret_cast<cx<T> *>(a.psi) + (((long)inst * 2 + pl.comp) * a.ny + y) * N;
#pragma unroll
    for (int m = 0; m < E; ++m) p[pl.t + m * TT] = v[0][m];
    __syncthreads();  // every thread is done with buffer s
    if (threadIdx.x == 0) {
      const int nt = tile + kPipe * gridDim.x;
      if (nt < ntiles) {
        fence_proxy_async();
        issue(nt, s);
      }
    }
  }
}


// Columns per tile of the persistent column pass: a 128-byte row segment
// where two tile buffers fit in about 110 KB and the block stays within 512
// threads; at least 16 bytes (one TMA row of 8-byte elements).
template <class T> __host__ __device__ constexpr int colp_cols_c(int logn, int loge) {
  const int n = 1 << logn, tt = n >> loge, es = (int)sizeof(cx<T>);
  int c = 128 / es;
  while (c > 1 && (c * tt > kColMaxThreads || kPipe * colp_buf_bytes(n, c, es) > 112 * 1024)) c /= 2;
  if (c * es < 16) c = 16 / es;
  return c;
}

template <class T, int LOGN, int LOGE, bool IMAG, int C>
__global__ void __launch_bounds__(LOGN <= 8 ? 256 : 512, LOGN <= 8 ? 2 : 1)
    col_pass_p(const __grid_constant__ CUtensorMap map, const ColArgs a, int ntiles) {
  constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
  constexpr int ES = sizeof(cx<T>);
  constexpr int XMUL = ES / 8;             // tensor-map elements per complex value
  constexpr int BOXH = N < 256 ? N : 256;  // rows per TMA box
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr size_t bufb = colp_buf_bytes(N, C, ES);
  cx<T> *btab = reinterpret_cast<cx<T> *>(smem_raw + kPipe * bufb);
  uint64_t *bar = reinterpret_cast<uint64_t *>(btab + N);
  const int c = threadIdx.x % C, t = threadIdx.x / C;
  const int cgroups = a.nx / C;
  const uint32_t tilebytes = (uint32_t)N * C * ES;

  auto buf = [&](int s) { return reinterpret_cast<cx<T> *>(smem_raw + s * bufb); };
  auto issue = [&](int tile, int s) {
    const int pc = tile / cgroups, cg = tile - pc * cgroups;
    mbar_expect_tx(&bar[s], tilebytes);
    for (int h = 0; h < N; h += BOXH) tma_g2s_2d(buf(s) + h * C, &map, cg * C * XMUL, pc * N + h, &bar[s]);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kPipe; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
    for (int s = 0; s < kPipe; ++s)
      if (blockIdx.x + s * gridDim.x < ntiles) issue(blockIdx.x + s * gridDim.x, s);
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) btab[k] = reinterpret_cast<const cx<T> *>(a.kyt)[k];
  __syncthreads();
  T inv;
  if constexpr (sizeof(T) == 4) inv = a.inv_f; else inv = a.inv_d;

  int i = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    const int s = i % kPipe;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((i / kPipe) & 1));
    if (!__syncthreads_and(ok)) {
      drain_after_timeout(bar, i, tile, ntiles, a.flags);
      return;
    }
    const int pc = tile / cgroups, kx = (tile - pc * cgroups) * C + c;
    cx<T> *b = buf(s);
    cx<T> v[1][E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[0][m] = b[(t + m * TT) * C + c];
    const cx<T> am = reinterpret_cast<const cx<T> *>(a.kxt)[(long)pc * a.nx + kx];
    __syncthreads();  // the dense tile is read; its space now serves the exchanges
    const ColAccC<T, C> acc{b + c};
    col_compute<T, LOGN, LOGE, IMAG>(v, t, acc, a.tw, am, btab, inv);
    cx<T> *col = reinterpret_cast<cx<T> *>(a.psi) + (long)pc * N * a.nx + kx;
    const int rs = TT * a.nx;
#pragma unroll
    for (int m = 0; m < E; ++m) col[t * a.nx + m * rs] = v[0][m];
    __syncthreads();  // every thread is done with buffer s
    if (threadIdx.x == 0) {
      const int nt = tile + kPipe * gridDim.x;
      if (nt < ntiles) {
        fence_proxy_async();
        issue(nt, s);
      }
    }
  }
}

}  // namespace spgpe
