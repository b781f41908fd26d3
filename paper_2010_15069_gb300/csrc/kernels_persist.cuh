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

// ------------------------------------------------ persistent row pass
//
// The rows are handed out in units: a warp's worth of rows when a row lies
// within one warp (2*TT <= 32 threads), else one row per block.  Each unit
// owns a staging buffer, an exchange area and an mbarrier in shared memory and
// loops over its rows; while it transforms one group of rows, the next group
// is already streaming into its staging buffer (two bulk copies, one per
// component, issued by the unit's first thread).  A warp unit synchronises
// with warp barriers only, so the warps of a block never wait for one another.

template <int N, int E> struct RowUnit {
  static constexpr int TT = N / E;
  static constexpr bool WARP = row_warp_local(TT);
  static constexpr int ROWS = WARP ? 32 / (2 * TT) : 1;      // rows per unit
  static constexpr int THREADS = WARP ? 32 : 2 * TT;         // threads per unit
};

// Shared-memory bytes of one unit: staging (rows x 2 components x n), then
// the exchange area (rows x row_stride), then the mbarrier; 128-byte aligned.
__host__ __device__ constexpr size_t rowu_bytes(int n, int rows, int es) {
  return ((size_t)rows * 2 * n * es + (size_t)rows * row_stride(n, es) * es + 8 + 127) / 128 * 128;
}

// Atom-number partials of one warp unit (its rows belong to one instance),
// in two halves so that the count's round trip overlaps the unit's stores:
// warp_partials_post adds the lanes' values in a fixed tree in the working
// precision (FP32 for complex64: non-negative summands, relative error below
// 13 units of FP32 rounding for 8 points per lane), lane 0 writes the unit's
// pair in FP64 and counts the unit (release-acquire), returning the count
// before it; warp_partials_finish lets the last unit of the instance reduce
// all pairs in a fixed order (FP64) and write the renormalisation scale, as
// row_partials does for blocks.
template <class T>
__device__ __forceinline__ unsigned warp_partials_post(const RowArgs &a, int inst, int group, int ngroups,
                                                       T (&tsum)[2]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tsum[0] += __shfl_xor_sync(0xffffffffu, tsum[0], o);
    tsum[1] += __shfl_xor_sync(0xffffffffu, tsum[1], o);
  }
  unsigned prev = 0;
  if ((threadIdx.x & 31) == 0) {
    if (in_bounds(a.flags, ((long)inst * ngroups + group) * 2 + 1, (long)a.ninst * a.ny * 2) &&
        in_bounds(a.flags, inst, a.ninst)) {
      a.partials[((long)inst * ngroups + group) * 2] = double(tsum[0]);
      a.partials[((long)inst * ngroups + group) * 2 + 1] = double(tsum[1]);
    }
    prev = count_group(&a.counters[inst]);
  }
  return prev;
}

template <class T>
__device__ __forceinline__ void warp_partials_finish(const RowArgs &a, int inst, int ngroups, unsigned prev) {
  const int lane = threadIdx.x & 31;
  prev = __shfl_sync(0xffffffffu, prev, 0);
  if (prev != (unsigned)ngroups - 1u) return;
  __threadfence();
  double tot[2] = {0.0, 0.0};
  for (int b = lane; b < ngroups; b += 32) {
    tot[0] += __ldcg(&a.partials[((long)inst * ngroups + b) * 2]);
    tot[1] += __ldcg(&a.partials[((long)inst * ngroups + b) * 2 + 1]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot[0] += __shfl_xor_sync(0xffffffffu, tot[0], o);
    tot[1] += __shfl_xor_sync(0xffffffffu, tot[1], o);
  }
  if (lane == 0) {
    const double nu = tot[0] * a.wgt, nd = tot[1] * a.wgt;
    double s0, s1;
    if (a.norm_mode == 1) {
      s0 = sqrt(a.tgt0 / nu);
      s1 = sqrt(a.tgt1 / nd);
    } else {
      s0 = s1 = sqrt((a.tgt0 + a.tgt1) / (nu + nd));
    }
    if (!isfinite(s0) || !isfinite(s1)) atomicOr(a.flags, 1);
    write_scale<T>(a, inst, s0, s1);
  }
}

// Warp units: blocks of SPGPE_ROWU_WARPS warps, SPGPE_ROWU_MINB of them
// resident per SM (the register budget; 8 x 3 measured fastest on GB300 at
// 256^2, ahead of 4 x 5, 10 x 2 and 20 x 1, and ahead of variants whose warps
// meet at a block barrier before every row group).  Otherwise one row of
// 2*TT threads per block.
#ifndef SPGPE_ROWU_WARPS
#define SPGPE_ROWU_WARPS 8
#endif
#ifndef SPGPE_ROWU_MINB
#define SPGPE_ROWU_MINB 3
#endif
__host__ __device__ constexpr int rowu_block(int n, int e) {
  return row_warp_local(n / e) ? 32 * SPGPE_ROWU_WARPS : 2 * (n / e);
}
// Dynamic shared memory of a block: its units, then (warp units only) a copy
// of the x plan's twiddle table.
__host__ __device__ constexpr size_t rowu_smem(int n, int e, int es, int tw_entries) {
  return row_warp_local(n / e) ? (size_t)(rowu_block(n, e) / 32) * rowu_bytes(n, 32 / (2 * (n / e)), es) +
                                     (size_t)tw_entries * 16
                               : rowu_bytes(n, 1, es);
}
// Resident blocks the register budget is sized for: 24 warps per SM for
// single-precision warp units, SPGPE_ROWB_THREADS_SP threads per SM for
// single-precision block units (640: 96 registers a thread), 16 warps in
// double precision.
#ifndef SPGPE_ROWB_THREADS_SP
#define SPGPE_ROWB_THREADS_SP 640
#endif
__host__ __device__ constexpr int rowu_min_blocks(int n, int e, int es) {
  return row_warp_local(n / e) && es == 8 ? SPGPE_ROWU_MINB
         : (es == 8 ? SPGPE_ROWB_THREADS_SP : 512) / rowu_block(n, e) > 0
             ? (es == 8 ? SPGPE_ROWB_THREADS_SP : 512) / rowu_block(n, e)
             : 1;
}

template <class T, int LOGN, int LOGE, int F>
__global__ void __launch_bounds__(rowu_block(1 << LOGN, 1 << LOGE),
                                  rowu_min_blocks(1 << LOGN, 1 << LOGE, sizeof(cx<T>)))
    row_pass_p(const RowArgs a, int nunits) {
  constexpr int N = 1 << LOGN, E = 1 << LOGE, TT = N / E;
  constexpr int ES = sizeof(cx<T>);
  using U = RowUnit<N, E>;
  constexpr int RU = U::ROWS, PADN = row_pad_n(N, ES), RS = row_stride(N, ES);
  constexpr size_t UB = rowu_bytes(N, RU, ES);
  constexpr uint32_t CB = (uint32_t)RU * N * ES;  // bytes of one component of a unit
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // Placement (as row_place, with blockDim >= 32 known here): lanes 0-15 of a
  // warp hold component up, lanes 16-31 component down.
  const int tx = threadIdx.x;
  const int comp = (tx >> 4) & 1;
  const int tp = (tx & 15) + 16 * (tx >> 5);
  const int slot = U::WARP ? (tx >> 5) : 0;
  const int lrow = tp / TT - slot * RU;  // row within the unit
  const int t = tp % TT;
  const int units_per_block = U::WARP ? (int)(blockDim.x >> 5) : 1;
  unsigned char *ub = smem_raw + slot * UB;
  cx<T> *stage = reinterpret_cast<cx<T> *>(ub);
  uint64_t *bar = reinterpret_cast<uint64_t *>(ub + UB - 8);
  const bool leader = U::WARP ? (tx & 31) == 0 : tx == 0;
  const int upi = a.ny / RU;  // units per instance
  auto sync_unit = [&] {
    if constexpr (U::WARP) __syncwarp(); else __syncthreads();
  };
  auto issue = [&](int u) {
    const int inst = u / upi, y0 = (u - inst * upi) * RU;
    const cx<T> *src = reinterpret_cast<const cx<T> *>(a.psi) + ((long)inst * 2 * a.ny + y0) * N;
    // (bounds-checked build: the last element of the second copy lies within psi)
    in_bounds(a.flags, ((long)inst * 2 * a.ny + y0) * N + (long)a.ny * N + RU * N - 1, (long)a.ninst * 2 * a.ny * N);
    mbar_expect_tx(bar, 2 * CB);
    bulk_g2s(stage, src, CB, bar);
    bulk_g2s(stage + RU * N, src + (long)a.ny * N, CB, bar);
  };

  // warp units read the twiddles from a shared-memory copy of the table
  using TwT = typename TwType<T>::type;
  constexpr int TWN = Plan<LOGN, LOGE>::entries();
  const TwT *tw = reinterpret_cast<const TwT *>(a.tw);
  if constexpr (U::WARP) {
    TwT *tws = reinterpret_cast<TwT *>(smem_raw + units_per_block * UB);
    for (int k = tx; k < TWN; k += blockDim.x) tws[k] = tw[k];
    __syncthreads();
    tw = tws;
  }
  RowArgs ac = a;
  ac.tw = tw;

  const int ustride = gridDim.x * units_per_block;
  // the first unit at or after v (in steps of ustride) whose instance is not frozen
  auto next_active = [&](int v) {
    if (a.active)
      while (v < nunits && !a.active[v / upi]) v += ustride;
    return v;
  };
  int u = next_active(blockIdx.x * units_per_block + slot);
  if (leader) {
    mbar_init(bar, 1);
    mbar_fence_init();
    if (u < nunits) issue(u);
  }
  sync_unit();
  const RowAcc<T, U::WARP> acc{stage + 2 * RU * N + lrow * RS + comp * PADN, 0, 0xffffffffu};
  const cx<T> *mine = stage + (comp * RU + lrow) * N + t;
#pragma unroll 1
  for (int it = 0; u < nunits; ++it) {
    // the leader waits for the copy; the unit's barrier orders the other
    // threads' reads after that wait and passes the outcome on
    bool ok = true;
    if (leader) ok = mbar_wait_bounded(bar, (uint32_t)(it & 1));
    if constexpr (U::WARP) {
      __syncwarp();
      ok = __shfl_sync(0xffffffffu, ok, 0);
    } else {
      ok = __syncthreads_or(!ok) == 0;
    }
    if (!ok) {
      // the copy for u may still land: give it one more bounded wait before leaving
      if (leader) {
        atomicOr(a.flags, kErrTimeout);
        mbar_wait_bounded(bar, (uint32_t)(it & 1));
      }
      return;
    }
    cx<T> v[1][E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[0][m] = mine[m * TT];
    sync_unit();  // the staging buffer is read: refill it with the next rows
    const int un = next_active(u + ustride);
    if (leader && un < nunits) {
      fence_proxy_async();
      issue(un);
    }
    const int inst = u / upi, group = u - inst * upi;
    const int y = group * RU + lrow;
    T nsum[2] = {T(0), T(0)};
    row_compute<T, LOGN, LOGE, F>(v, t, comp, 0xffffffffu, 16, inst, y, acc,
                                  reinterpret_cast<const q4<T> *>(a.tabx) + (long)inst * N, ac, nsum);
    unsigned prev = 0;
    if constexpr (F & F_PART) {
      if constexpr (U::WARP) prev = warp_partials_post<T>(a, inst, group, upi, nsum);
      else row_partials<T>(a, inst, group, upi, nsum);
    }
    cx<T> *p = reinterpret_cast<cx<T> *>(a.psi) + (((long)inst * 2 + comp) * a.ny + y) * N + t;
    const long pb = (((long)inst * 2 + comp) * a.ny + y) * N + t, pt = (long)a.ninst * 2 * a.ny * N;
#pragma unroll
    for (int m = 0; m < E; ++m)
      if (in_bounds(a.flags, pb + m * TT, pt)) p[m * TT] = v[0][m];
    if constexpr ((F & F_PART) && U::WARP) warp_partials_finish<T>(a, inst, upi, prev);
    u = un;
  }
}

// Columns per tile of the persistent column pass: a 128-byte row segment
// where two tile buffers fit in about 110 KB (160 KB for columns of 2048 rows
// or more, which run one block per SM) and the block stays within 512
// threads; at least 16 bytes (one TMA row of 8-byte elements).
template <class T> __host__ __device__ constexpr int colp_cols_c(int logn, int loge) {
  const int n = 1 << logn, tt = n >> loge, es = (int)sizeof(cx<T>);
  const size_t cap = (logn >= 11 ? 160 : 112) * 1024;
  int c = 128 / es;
  while (c > 1 && (c * tt > kColMaxThreads || kPipe * colp_buf_bytes(n, c, es) > cap)) c /= 2;
  if (c * es < 16) c = 16 / es;
  return c;
}

// Bytes of the column plan's twiddle table the persistent column pass keeps
// in shared memory: the whole table when the block's shared memory (two tile
// buffers, the K table, the table, the barriers) stays within a block's
// limit (in complex64 columns of up to 2048 rows), else none (the table
// stays in global memory).
template <class T> __host__ __device__ constexpr size_t colp_tw_bytes(int logn, int c, int entries) {
  return kPipe * colp_buf_bytes(1 << logn, c, (int)sizeof(cx<T>)) + ((size_t)1 << logn) * sizeof(cx<T>) +
                     (size_t)entries * sizeof(typename TwType<T>::type) + kPipe * sizeof(uint64_t) <=
                 kMaxSmemPerBlock
             ? (size_t)entries * sizeof(typename TwType<T>::type)
             : 0;
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
  using TwT = typename TwType<T>::type;
  constexpr int TWN = Plan<LOGN, LOGE>::entries();
  constexpr size_t TWB = colp_tw_bytes<T>(LOGN, C, TWN);
  cx<T> *btab = reinterpret_cast<cx<T> *>(smem_raw + kPipe * bufb);
  TwT *tws = reinterpret_cast<TwT *>(btab + N);
  uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(tws) + TWB);
  const int c = threadIdx.x % C, t = threadIdx.x / C;
  const int cgroups = a.nx / C;
  const uint32_t tilebytes = (uint32_t)N * C * ES;

  auto buf = [&](int s) { return reinterpret_cast<cx<T> *>(smem_raw + s * bufb); };
  auto issue = [&](int tile, int s) {
    const int pc = tile / cgroups, cg = tile - pc * cgroups;
    // (bounds-checked build: the boxes lie within the tensor map)
    in_bounds(a.flags, (long)(cg + 1) * C * XMUL - 1, (long)a.nx * XMUL);
    in_bounds(a.flags, (long)pc * N + N - 1, (long)a.ninst * 2 * N);
    mbar_expect_tx(&bar[s], tilebytes);
    for (int h = 0; h < N; h += BOXH) tma_g2s_2d(buf(s) + h * C, &map, cg * C * XMUL, pc * N + h, &bar[s]);
  };

  // the first tile at or after v (in steps of gridDim.x) whose instance is not frozen
  auto next_active = [&](int v) {
    if (a.active)
      while (v < ntiles && !a.active[v / (2 * cgroups)]) v += gridDim.x;
    return v;
  };
  // the tile being processed (buffer i % 2) and the one streaming into the
  // other buffer (ntiles: none)
  static_assert(kPipe == 2, "two tile buffers");
  int tile = next_active(blockIdx.x);
  int nxt = tile < ntiles ? next_active(tile + gridDim.x) : ntiles;
  if (threadIdx.x == 0) {
    for (int q = 0; q < kPipe; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
    if (tile < ntiles) issue(tile, 0);
    if (nxt < ntiles) issue(nxt, 1);
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) btab[k] = reinterpret_cast<const cx<T> *>(a.kyt)[k];
  const void *tw = a.tw;
  if constexpr (TWB > 0) {
    for (int k = threadIdx.x; k < TWN; k += blockDim.x) tws[k] = reinterpret_cast<const TwT *>(a.tw)[k];
    tw = tws;
  }
  __syncthreads();

  for (int i = 0; tile < ntiles; ++i) {
    const int s = i & 1;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((i >> 1) & 1));
    if (!__syncthreads_and(ok)) {
      // a wait ran out: record it, and give the copy still in flight into the
      // other buffer (if any) its own bounded wait before leaving
      if (threadIdx.x == 0) {
        atomicOr(a.flags, kErrTimeout);
        if (nxt < ntiles) mbar_wait_bounded(&bar[s ^ 1], (uint32_t)(((i + 1) >> 1) & 1));
      }
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
    col_compute<T, LOGN, LOGE, IMAG>(v, t, acc, tw, am, btab, col_inv<T>(a, pc));
    cx<T> *col = reinterpret_cast<cx<T> *>(a.psi) + (long)pc * N * a.nx + kx;
    const int rs = TT * a.nx;
    const long cb = (long)pc * N * a.nx + kx, ct = (long)a.ninst * 2 * N * a.nx;
#pragma unroll
    for (int m = 0; m < E; ++m)
      if (in_bounds(a.flags, cb + t * a.nx + m * rs, ct)) col[t * a.nx + m * rs] = v[0][m];
    __syncthreads();  // every thread is done with buffer s
    // refill buffer s with the tile after the one waiting in the other buffer
    const int after = nxt < ntiles ? next_active(nxt + gridDim.x) : ntiles;
    if (threadIdx.x == 0 && after < ntiles) {
      fence_proxy_async();
      issue(after, s);
    }
    tile = nxt;
    nxt = after;
  }
}

// ------------------------------------ warp-local column pass (256 rows, c64)
//
// Tiles of 16 columns x 256 rows of one component arrive by TMA with the
// 128-byte swizzle: row r of a tile is one 128-byte line whose 16-byte chunks
// (two columns each) are permuted by chunk ^ (r & 7).  Each warp owns two
// adjacent columns; its lane l holds column 2w + ((l >> 3) & 1) at positions
// t + 16 m, t = (l & 7) + 8 (l >> 4), so each half-warp touches 8 consecutive
// rows of both columns: all 32 banks once, for the tile reads and the result
// writes alike.  The FFT exchanges run in a per-warp padded area (column
// stride 280 elements, one pad per 16) under warp barriers only; the results
// go back into the tile in place and leave by one TMA store of the tile.  Per
// tile the block meets two barriers: after the load lands, before the store.

constexpr int kColW_C = 16, kColW_N = 256, kColW_TT = 16;
constexpr int kColW_XS = 280;  // exchange elements per column (256 + 16 pads + 8 bank shift)
constexpr size_t kColW_Tile = (size_t)kColW_N * kColW_C * 8;  // 32 KiB, 1 KiB aligned

__host__ __device__ constexpr size_t colw_smem() {
  return 1024 + 128 /* alignment slack, margin */ + 2 * kColW_Tile + (size_t)8 * 2 * kColW_XS * 8 + kColW_N * 8 + 2 * 8;
}

struct ColAccW {
  cx<float> *base;  // this column's exchange area
  __device__ __forceinline__ void st(int, int p, cx<float> v) const { base[p + (p >> 4)] = v; }
  __device__ __forceinline__ cx<float> ld(int, int p) const { return base[p + (p >> 4)]; }
  __device__ __forceinline__ static void sync() { __syncwarp(); }
};

// byte offset of (row r, column c) in a swizzled tile
__device__ __forceinline__ uint32_t sw_off(int r, int c) {
  return (uint32_t)r * 128u + ((uint32_t)((c >> 1) ^ (r & 7)) << 4) + ((uint32_t)(c & 1) << 3);
}

template <bool IMAG>
__global__ void __launch_bounds__(256, 2)
    col_pass_w(const __grid_constant__ CUtensorMap map, const ColArgs a, int ntiles) {
  constexpr int N = kColW_N, E = 16, TT = kColW_TT, C = kColW_C;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *tiles = sm;
  cx<float> *xch = reinterpret_cast<cx<float> *>(sm + 2 * kColW_Tile);
  cx<float> *btab = xch + 8 * 2 * kColW_XS;
  uint64_t *bar = reinterpret_cast<uint64_t *>(btab + N);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cl = (lane >> 3) & 1;                 // column within the warp's pair
  const int c = 2 * w + cl;                       // column within the tile
  const int t = (lane & 7) + 8 * (lane >> 4);     // position index within the column
  const int cgroups = a.nx / C;
  const ColAccW acc{xch + (w * 2 + cl) * kColW_XS};

  auto next_active = [&](int v) {
    if (a.active)
      while (v < ntiles && !a.active[v / (2 * cgroups)]) v += gridDim.x;
    return v;
  };
  auto issue = [&](int tile, int s) {
    const int pc = tile / cgroups, cg = tile - pc * cgroups;
    // (bounds-checked build: the box lies within the tensor map)
    in_bounds(a.flags, (long)(cg + 1) * C - 1, a.nx);
    in_bounds(a.flags, (long)pc * N + N - 1, (long)a.ninst * 2 * N);
    mbar_expect_tx(&bar[s], (uint32_t)kColW_Tile);
    tma_g2s_2d(tiles + s * kColW_Tile, &map, cg * C, pc * N, &bar[s]);
  };
  int tile = next_active(blockIdx.x);
  int nxt = tile < ntiles ? next_active(tile + gridDim.x) : ntiles;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
    if (tile < ntiles) issue(tile, 0);
    if (nxt < ntiles) issue(nxt, 1);
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) btab[k] = reinterpret_cast<const cx<float> *>(a.kyt)[k];
  __syncthreads();
  int refill = ntiles, refill_s = 0;  // a buffer whose store must finish reading before its reload
  for (int i = 0; tile < ntiles; ++i) {
    const int s = i & 1;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((i >> 1) & 1));
    if (!__syncthreads_and(ok)) {
      // loads still in flight: this buffer's, and the other's on the first
      // tile only (later reloads of the other buffer are not yet issued here)
      if (threadIdx.x == 0) {
        atomicOr(a.flags, kErrTimeout);
        mbar_wait_bounded(&bar[s], (uint32_t)((i >> 1) & 1));
        if (nxt < ntiles && refill == ntiles) mbar_wait_bounded(&bar[s ^ 1], (uint32_t)(((i + 1) >> 1) & 1));
        bulk_wait0();
      }
      return;
    }
    // the previous tile's store has had this tile's wait to read its buffer
    if (threadIdx.x == 0 && refill < ntiles) {
      bulk_wait_read0();
      issue(refill, refill_s);
    }
    refill = ntiles;    unsigned char *tb = tiles + s * kColW_Tile;
    const int pc = tile / cgroups, kx = (tile - pc * cgroups) * C + c;
    cx<float> v[1][E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[0][m] = *reinterpret_cast<const cx<float> *>(tb + sw_off(t + m * TT, c));
    const cx<float> am = reinterpret_cast<const cx<float> *>(a.kxt)[(long)pc * a.nx + kx];
    col_compute<float, 8, 4, IMAG>(v, t, acc, a.tw, am, btab, col_inv<float>(a, pc));
    // results in place (this warp's columns only), then one store of the tile
#pragma unroll
    for (int m = 0; m < E; ++m) *reinterpret_cast<cx<float> *>(tb + sw_off(t + m * TT, c)) = v[0][m];
    fence_proxy_async();
    __syncthreads();
    const int after = nxt < ntiles ? next_active(nxt + gridDim.x) : ntiles;
    if (threadIdx.x == 0) {
      const int cg = tile - pc * cgroups;
      in_bounds(a.flags, (long)(cg + 1) * C - 1, a.nx);
      in_bounds(a.flags, (long)pc * N + N - 1, (long)a.ninst * 2 * N);
      tma_s2g_2d(&map, cg * C, pc * N, tb);
      bulk_commit();
    }
    // buffer s is reloaded (with `after`, which exists only if nxt does) once
    // its store has read it: at the next tile's start
    if (after < ntiles) {
      refill = after;
      refill_s = s;
    }
    tile = nxt;
    nxt = after;
  }
  if (threadIdx.x == 0) bulk_wait0();
}

}  // namespace spgpe
