// Column-pass, energy and reduction launchers (included once per precision by
// kernels_col_f32.cu / kernels_col_f64.cu).
#pragma once
#include <algorithm>

#include "kernels_persist.cuh"

namespace spgpe {

template <class T> constexpr int col_loge(int logn) { return col_loge_for(logn, sizeof(cx<T>)); }

template <class T> LaunchShape col_shape(int nx, int ny) {
  int logn = 0;
  while ((1 << logn) < ny) ++logn;
  const int E = 1 << col_loge<T>(logn);
  const int TT = ny / E;
  const int cmax = 128 / (int)sizeof(cx<T>);  // one 128-byte line of a row
  const int C = std::max(1, std::min(std::min(cmax, nx), kColMaxThreads / TT));
  LaunchShape s;
  s.elems_per_thread = E;
  s.threads = C * TT;
  s.blocks_x = nx / C;
  s.rows_or_cols = C;
  s.smem = (size_t)col_smem_elems(ny, C, sizeof(cx<T>)) * sizeof(cx<T>);
  return s;
}

template <class K> cudaError_t grant_smem_c(K kern, size_t smem, int &granted) {
  if ((int)smem > granted) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    granted = (int)smem;
  }
  return cudaSuccess;
}

template <class T, int LOGN, bool IMAG> cudaError_t col_launch_n(ColArgs a, cudaStream_t st) {
  constexpr int LOGE = col_loge<T>(LOGN);
  auto kern = col_pass<T, LOGN, LOGE, IMAG>;
  const LaunchShape sh = col_shape<T>(a.nx, a.ny);
  static int granted = 0;
  cudaError_t e = grant_smem_c(kern, sh.smem, granted);
  if (e != cudaSuccess) return e;
  a.C = sh.rows_or_cols;
  kern<<<dim3(sh.blocks_x, 2, a.ninst), sh.threads, sh.smem, st>>>(a);
  return cudaGetLastError();
}

template <class T, int LOGN> cudaError_t energy_launch_n(EnergyArgs a, cudaStream_t st, int *rb, int *cb) {
  // row part: the row-pass geometry
  {
    constexpr int LOGE = erow_loge_for(LOGN, sizeof(cx<T>));
    auto kern = energy_row<T, LOGN, LOGE>;
    const int E = 1 << LOGE;
    const int TT = a.nx / E;
    const int rows = std::max(1, std::min(kRowMaxThreads / TT, a.ny));
    const size_t smem = (size_t)rows * row_stride(a.nx, sizeof(cx<T>)) * sizeof(cx<T>);
    static int granted = 0;
    cudaError_t e = grant_smem_c(kern, smem, granted);
    if (e != cudaSuccess) return e;
    a.rows = rows;
    *rb = a.ny / rows;
    kern<<<dim3(a.ny / rows, a.ninst), rows * TT, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class T, int LOGN> cudaError_t energy_col_launch_n(EnergyArgs a, cudaStream_t st, int *cb) {
  constexpr int LOGE = col_loge<T>(LOGN);
  auto kern = energy_col<T, LOGN, LOGE>;
  const LaunchShape sh = col_shape<T>(a.nx, a.ny);
  static int granted = 0;
  cudaError_t e = grant_smem_c(kern, sh.smem, granted);
  if (e != cudaSuccess) return e;
  a.C = sh.rows_or_cols;
  *cb = sh.blocks_x;
  kern<<<dim3(sh.blocks_x, 2, a.ninst), sh.threads, sh.smem, st>>>(a);
  return cudaGetLastError();
}

#define SPGPE_SWITCH_LOGN(n, CALL)  \
  switch (n) {                      \
    case 8: return CALL(3);         \
    case 16: return CALL(4);        \
    case 32: return CALL(5);        \
    case 64: return CALL(6);        \
    case 128: return CALL(7);       \
    case 256: return CALL(8);       \
    case 512: return CALL(9);       \
    case 1024: return CALL(10);     \
    case 2048: return CALL(11);     \
    case 4096: return CALL(12);     \
    default: return cudaErrorInvalidValue; \
  }

template <class T> cudaError_t launch_col(bool imag, ColArgs a, cudaStream_t st) {
#define SPGPE_COL_REAL(L) col_launch_n<T, L, false>(a, st)
#define SPGPE_COL_IMAG(L) col_launch_n<T, L, true>(a, st)
  if (imag) {
    SPGPE_SWITCH_LOGN(a.ny, SPGPE_COL_IMAG)
  } else {
    SPGPE_SWITCH_LOGN(a.ny, SPGPE_COL_REAL)
  }
#undef SPGPE_COL_REAL
#undef SPGPE_COL_IMAG
}

template <class T> cudaError_t launch_energy_rows(EnergyArgs a, cudaStream_t st, int *rb) {
#define SPGPE_EROW(L) energy_launch_n<T, L>(a, st, rb, nullptr)
  SPGPE_SWITCH_LOGN(a.nx, SPGPE_EROW)
#undef SPGPE_EROW
}

template <class T> cudaError_t launch_energy_cols(EnergyArgs a, cudaStream_t st, int *cb) {
#define SPGPE_ECOL(L) energy_col_launch_n<T, L>(a, st, cb)
  SPGPE_SWITCH_LOGN(a.ny, SPGPE_ECOL)
#undef SPGPE_ECOL
}

// Both energy passes.  The caller sizes a.partials for the row part and gets
// the block counts back; the column part writes behind the row partials.
template <class T> cudaError_t launch_energy(EnergyArgs a, cudaStream_t st, int *row_blocks, int *col_blocks) {
  cudaError_t e = launch_energy_rows<T>(a, st, row_blocks);
  if (e != cudaSuccess) return e;
  EnergyArgs b = a;
  b.partials = a.partials + (long)a.ninst * (*row_blocks) * 6;
  return launch_energy_cols<T>(b, st, col_blocks);
}

template <class T> cudaError_t launch_norm(const void *psi, long plane, int ninst, double *partials, int blocks,
                                           cudaStream_t st) {
  norm_kernel<T><<<dim3(blocks, ninst), 256, 0, st>>>(reinterpret_cast<const cx<T> *>(psi), plane, partials);
  return cudaGetLastError();
}

template <class T> cudaError_t launch_residual(const void *psi, const void *prev, long plane, int ninst,
                                               double *partials, int blocks, cudaStream_t st) {
  residual_kernel<T><<<dim3(blocks, ninst), 256, 0, st>>>(reinterpret_cast<const cx<T> *>(psi),
                                                          reinterpret_cast<const cx<T> *>(prev), plane, partials);
  return cudaGetLastError();
}

// ---- persistent column pass

template <class T> int colp_cols(int nx, int ny) {
  int logn = 0;
  while ((1 << logn) < ny) ++logn;
  return colp_cols_c<T>(logn, col_loge<T>(logn));
}

template <class T, int LOGN, bool IMAG>
cudaError_t colp_launch_n(ColArgs a, const CUtensorMap &map, cudaStream_t st, int sms) {
  constexpr int LOGE = col_loge<T>(LOGN);
  constexpr int N = 1 << LOGN, TT = N >> LOGE;
  constexpr int C = colp_cols_c<T>(LOGN, LOGE);
  if (a.nx < C) return cudaErrorNotSupported;  // narrower than one tile: the plain pass
  auto kern = col_pass_p<T, LOGN, LOGE, IMAG, C>;
  const int threads = C * TT;
  const int es = sizeof(cx<T>);
  const size_t smem = kPipe * colp_buf_bytes(N, C, es) + (size_t)N * es +
                      colp_tw_bytes<T>(LOGN, C, Plan<LOGN, LOGE>::entries()) + kPipe * sizeof(uint64_t);
  if (smem > kMaxSmemPerBlock) return cudaErrorNotSupported;  // caller falls back to the plain pass
  static int granted = 0;
  cudaError_t e = grant_smem_c(kern, smem, granted);
  if (e != cudaSuccess) return e;
  static int occ_threads = -1, occ_blocks = 0;
  static size_t occ_smem = 0;
  if (occ_threads != threads || occ_smem != smem) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_blocks, kern, threads, smem);
    if (e != cudaSuccess) return e;
    occ_threads = threads;
    occ_smem = smem;
  }
  const int ntiles = (a.nx / C) * 2 * a.ninst;
  const int grid = std::max(1, std::min(ntiles, std::max(1, occ_blocks) * sms));
  a.C = C;
  kern<<<grid, threads, smem, st>>>(map, a, ntiles);
  return cudaGetLastError();
}

template <class T> cudaError_t launch_col_p(bool imag, ColArgs a, const CUtensorMap &map, cudaStream_t st,
                                            int sms) {
#define SPGPE_COLP_REAL(L) colp_launch_n<T, L, false>(a, map, st, sms)
#define SPGPE_COLP_IMAG(L) colp_launch_n<T, L, true>(a, map, st, sms)
  if (imag) {
    SPGPE_SWITCH_LOGN(a.ny, SPGPE_COLP_IMAG)
  } else {
    SPGPE_SWITCH_LOGN(a.ny, SPGPE_COLP_REAL)
  }
#undef SPGPE_COLP_REAL
#undef SPGPE_COLP_IMAG
}

// ---- warp-local column pass (ny = 256, complex64; psi viewed through a
// 128-byte-swizzled tensor map with 16 x 256 boxes)

template <bool IMAG> cudaError_t colw_launch(ColArgs a, const CUtensorMap &map, cudaStream_t st, int sms) {
  auto kern = col_pass_w<IMAG>;
  const size_t smem = colw_smem();
  static int granted = 0, occ = -1;  // per instantiation (per time direction)
  cudaError_t e = grant_smem_c(kern, smem, granted);
  if (e != cudaSuccess) return e;
  if (occ < 0 && (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem)) != cudaSuccess) return e;
  const int ntiles = (a.nx / kColW_C) * 2 * a.ninst;
  const int grid = std::max(1, std::min(ntiles, std::max(1, occ) * sms));
  a.C = kColW_C;
  kern<<<grid, 256, smem, st>>>(map, a, ntiles);
  return cudaGetLastError();
}

template <class T> cudaError_t launch_col_w(bool imag, ColArgs a, const CUtensorMap &map, cudaStream_t st, int sms) {
  if (sizeof(T) != 4 || a.ny != kColW_N || a.nx < kColW_C) return cudaErrorNotSupported;
  return imag ? colw_launch<true>(a, map, st, sms) : colw_launch<false>(a, map, st, sms);
}

template <class T> cudaError_t launch_ref_K(const ColArgs &a, cudaStream_t st) {
  const long plane = (long)a.nx * a.ny;
  ref_K_kernel<T><<<dim3((unsigned)((plane + 255) / 256), 2 * a.ninst), 256, 0, st>>>(a);
  return cudaGetLastError();
}

#define SPGPE_INSTANTIATE_COL(T)                                                              \
  template LaunchShape col_shape<T>(int, int);                                                \
  template cudaError_t launch_col<T>(bool, ColArgs, cudaStream_t);                            \
  template cudaError_t launch_energy<T>(EnergyArgs, cudaStream_t, int *, int *);              \
  template cudaError_t launch_norm<T>(const void *, long, int, double *, int, cudaStream_t);  \
  template cudaError_t launch_residual<T>(const void *, const void *, long, int, double *, int, \
                                          cudaStream_t);                                      \
  template cudaError_t launch_ref_K<T>(const ColArgs &, cudaStream_t);                      \
  template int colp_cols<T>(int, int);                                                        \
  template cudaError_t launch_col_p<T>(bool, ColArgs, const CUtensorMap &, cudaStream_t, int);     \
  template cudaError_t launch_col_w<T>(bool, ColArgs, const CUtensorMap &, cudaStream_t, int);

}  // namespace spgpe
