// Row-pass launchers (included once per precision by kernels_row_f32.cu /
// kernels_row_f64.cu).
#pragma once
#include <algorithm>

#include "kernels_persist.cuh"

namespace spgpe {

template <class T> constexpr int row_loge(int logn) { return row_loge_for(logn, sizeof(cx<T>)); }

template <class T> LaunchShape row_shape(int nx, int ny) {
  int logn = 0;
  while ((1 << logn) < nx) ++logn;
  const int E = 1 << row_loge<T>(logn);
  const int TT = nx / E;  // threads per component of a row
  const int rows = std::max(1, std::min(kRowMaxThreads / (2 * TT), ny));
  LaunchShape s;
  s.elems_per_thread = E;
  s.threads = 2 * rows * TT;
  s.blocks_x = ny / rows;
  s.rows_or_cols = rows;
  s.smem = (size_t)rows * row_stride(nx, sizeof(cx<T>)) * sizeof(cx<T>);
  return s;
}

template <class K> cudaError_t grant_smem(K kern, size_t smem, int &granted) {
  if ((int)smem > granted) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    granted = (int)smem;
  }
  return cudaSuccess;
}

template <class T, int LOGN, int F> cudaError_t row_launch_n(RowArgs a, cudaStream_t st) {
  constexpr int LOGE = row_loge<T>(LOGN);
  auto kern = row_pass<T, LOGN, LOGE, F>;
  const LaunchShape sh = row_shape<T>(a.nx, a.ny);
  static int attr_set = 0;  // largest dynamic shared memory granted so far
  if ((int)sh.smem > attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
    if (e != cudaSuccess) return e;
    attr_set = (int)sh.smem;
  }
  a.rows = sh.rows_or_cols;
  kern<<<dim3(sh.blocks_x, a.ninst), sh.threads, sh.smem, st>>>(a);
  return cudaGetLastError();
}

// One flag combination, every row length (instantiated per flag group in
// the kernels_row_*.cu units so that they compile in parallel).
template <class T, int F> cudaError_t launch_row_f(RowArgs a, cudaStream_t st) {
  switch (a.nx) {
    case 8: return row_launch_n<T, 3, F>(a, st);
    case 16: return row_launch_n<T, 4, F>(a, st);
    case 32: return row_launch_n<T, 5, F>(a, st);
    case 64: return row_launch_n<T, 6, F>(a, st);
    case 128: return row_launch_n<T, 7, F>(a, st);
    case 256: return row_launch_n<T, 8, F>(a, st);
    case 512: return row_launch_n<T, 9, F>(a, st);
    case 1024: return row_launch_n<T, 10, F>(a, st);
    case 2048: return row_launch_n<T, 11, F>(a, st);
    case 4096: return row_launch_n<T, 12, F>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---- persistent row pass

template <class T, int LOGN, int F> cudaError_t rowp_launch_n(RowArgs a, cudaStream_t st, int sms) {
  constexpr int LOGE = row_loge<T>(LOGN);
  constexpr int N = 1 << LOGN, E = 1 << LOGE;
  using U = RowUnit<N, E>;
  if (a.ny < U::ROWS) return cudaErrorNotSupported;  // a unit would span instances: the plain pass
  auto kern = row_pass_p<T, LOGN, LOGE, F>;
  const int threads = rowu_block(N, E);
  const int upb = U::WARP ? threads / 32 : 1;  // units per block
  const size_t smem = rowu_smem(N, E, sizeof(cx<T>), Plan<LOGN, LOGE>::entries());
  if (smem > kMaxSmemPerBlock) return cudaErrorNotSupported;
  static int granted = 0;
  cudaError_t e = grant_smem(kern, smem, granted);
  if (e != cudaSuccess) return e;
  static int occ_blocks = -1;
  if (occ_blocks < 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_blocks, kern, threads, smem);
    if (e != cudaSuccess) return e;
  }
  const int nunits = a.ninst * (a.ny / U::ROWS);
  const int grid = std::max(1, std::min((nunits + upb - 1) / upb, std::max(1, occ_blocks) * sms));
  a.rows = U::ROWS;
  kern<<<grid, threads, smem, st>>>(a, nunits);
  return cudaGetLastError();
}

template <class T, int F> cudaError_t launch_row_pf(RowArgs a, cudaStream_t st, int sms) {
  switch (a.nx) {
    case 8: return rowp_launch_n<T, 3, F>(a, st, sms);
    case 16: return rowp_launch_n<T, 4, F>(a, st, sms);
    case 32: return rowp_launch_n<T, 5, F>(a, st, sms);
    case 64: return rowp_launch_n<T, 6, F>(a, st, sms);
    case 128: return rowp_launch_n<T, 7, F>(a, st, sms);
    case 256: return rowp_launch_n<T, 8, F>(a, st, sms);
    case 512: return rowp_launch_n<T, 9, F>(a, st, sms);
    case 1024: return rowp_launch_n<T, 10, F>(a, st, sms);
    case 2048: return rowp_launch_n<T, 11, F>(a, st, sms);
    case 4096: return rowp_launch_n<T, 12, F>(a, st, sms);
    default: return cudaErrorInvalidValue;
  }
}

template <class T> cudaError_t launch_ref_R(bool imag, const RowArgs &a, cudaStream_t st) {
  const long plane = (long)a.nx * a.ny;
  const dim3 grid((unsigned)((plane + 255) / 256), a.ninst);
  if (imag) ref_R_kernel<T, true><<<grid, 256, 0, st>>>(a);
  else ref_R_kernel<T, false><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

#define SPGPE_INSTANTIATE_ROW_SHAPE(T)                                              \
  template LaunchShape row_shape<T>(int, int);                                      \
  template cudaError_t launch_ref_R<T>(bool, const RowArgs &, cudaStream_t);

#define SPGPE_INSTANTIATE_ROW_FLAG(T, F)                                            \
  template cudaError_t launch_row_f<T, F>(RowArgs, cudaStream_t);                   \
  template cudaError_t launch_row_pf<T, F>(RowArgs, cudaStream_t, int);

}  // namespace spgpe
