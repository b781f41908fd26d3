// Declarations shared by the kernel translation units and the C-ABI layer.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace spgpe {

// Row-pass work flags (one fused launch does the listed steps in order).
enum : int {
  F_IFFT = 1,     // load k_x-space row, inverse FFT along x
  F_REND = 2,     // R(dt/2) = X(dt/4) D(dt/2) X(dt/4): the step's closing half
  F_PART = 4,     // FP64 atom-number partials of the result; last block -> scale
  F_SCALE = 8,    // multiply by the per-instance scale (imaginary-time renormalisation)
  F_RSTART = 16,  // R(dt/2): the next step's opening half
  F_FFT = 32,     // forward FFT along x, store k_x-space row
  F_IMAG = 64,    // imaginary time: exp(-tau H) factors instead of exp(-i tau H)
  F_LAG = 128     // between R_end and R_start: multiply by the predicted scale (lagged renormalisation)
};

constexpr int kRealFirst = F_RSTART | F_FFT;
constexpr int kRealMid = F_IFFT | F_REND | F_RSTART | F_FFT;
constexpr int kRealLast = F_IFFT | F_REND;
constexpr int kImagFirst = F_IMAG | F_RSTART | F_FFT;
constexpr int kImagB = F_IMAG | F_SCALE | F_RSTART | F_FFT;
constexpr int kImagA = F_IMAG | F_IFFT | F_REND | F_PART;
constexpr int kImagScale = F_IMAG | F_SCALE;
// Lagged renormalisation (one row pass between steps): the step's closing
// R(dt/2), the atom-number partials of its result (the last unit writes the
// exact scale s_n), the scale predicted from the previous step (s_{n-1}), the
// next step's opening R(dt/2) and the x-FFT; the column pass that follows
// multiplies by s_n / s_{n-1}, so the linear part of the renormalisation is
// exact and only the densities seen by the opening D lag behind.
constexpr int kImagLag = F_IMAG | F_IFFT | F_REND | F_PART | F_LAG | F_RSTART | F_FFT;

// Arguments of the fused row pass (x direction, both components per thread).
struct RowArgs {
  void *psi;              // [ninst][2][ny][nx] complex, in place
  // step tables [ninst][nx], [ninst][ny]: {p(V+delta/2), p(V-delta/2), X constants}
  // of the separable pieces, p(v) = htau v (real time) or exp(-(dt/2) v)
  const void *tabx;
  const void *taby;
                          // (imaginary time: the factors exp(-tau (V +- delta/2)) of the
                          // separable pieces in place of the potentials)
                          // X constants: (tan(a/2), sin a) in real time, (cosh a - 1, sinh a)
                          // in imaginary time, a = Omega piece * dt / 8
  const void *pot2d;      // [ny][nx] {V+delta/2, V-delta/2, Omega, 0} or null
  const void *tw;         // twiddle table of the x plan (see TwType in fft_core.cuh)
  const double *gpar;     // [ninst][4] {g11, g22, g12, kL}
  const void *gparT;      // the same in the working precision
  double tau;             // D substep (dt/2)
  double xang;            // X(dt/4) rotation angle per unit Omega (dt/8)
  double htau_d;          // -tau/2 (real time, half phase) or -tau (imaginary time)
  float htau_f;           // the same in single precision
  float xang_f;           // xang in single precision
  int omega_pieces;       // bit 0: some Omega_y != 0, bit 1: some Omega_x != 0 (separable pieces)
  double *partials;       // [ninst][gridDim.x][2]
  unsigned *counters;     // [ninst], zero between launches
  double *scale;          // [ninst][2]: written by the last unit of F_PART
  void *scale_t;          // [ninst][2] the same in the working precision (read by F_SCALE)
  const double *scale_pred;    // [ninst][2]: the predicted scale of F_LAG (never the buffer written)
  const void *scale_pred_t;    // the same in the working precision (what F_LAG applies)
  void *cfac;             // [ninst][2] working precision, F_LAG only: the last unit writes
                          // scale / scale_pred, the column pass's correction (null otherwise)
  double tgt0, tgt1;      // target atom numbers
  int norm_mode;          // 0 total, 1 per component
  double wgt;             // dx * dy
  const int *active;      // [ninst] nonzero: step this instance (null: all); frozen instances are skipped
  int *flags;             // bit 0: non-finite or zero norm met
  int nx, ny, ninst, rows;
};

// Arguments of the fused column pass (y direction, one component per block).
struct ColArgs {
  void *psi;
  double inv_d;           // 1/(nx ny), an exact power of two
  float inv_f;
  int *flags;             // error bits (persistent pass: bit 1 = transfer wait timed out)
  const int *active;      // [ninst] as in RowArgs
  const void *kxt;        // [ninst][2][nx] complex a_j(kx) - 1
  const void *kyt;        // [ny] complex b(ky) - 1 (1/(nx ny) applied in the kernel)
  const void *tw;         // twiddle table of the y plan (see TwType in fft_core.cuh)
  // Lagged renormalisation: each column of instance i, component j is also
  // multiplied by cfac[2 i + j] (working precision: the exact scale over the
  // predicted one, written by the row pass before); null: no such factor.
  const void *cfac;
  int nx, ny, ninst, C;
};

// Energy passes.
struct EnergyArgs {
  const void *psi;
  void *scratch;          // [ninst][2][ny][nx] k_x-space copy
  const void *rawx;       // [ninst][nx] {Vx, delta_x, Omega_x, 0}
  const void *rawy;       // [ninst][ny] {Vy, delta_y, Omega_y, 0}
  const void *pot2d;      // [ny][nx] {V+delta/2, V-delta/2, Omega, 0} or null
  const void *twx, *twy;  // twiddle tables of the energy-row x plan and the column y plan
  const double *gpar;
  double *partials;       // row pass: [ninst][gridDim.x][6]; column pass: [ninst][2][gridDim.x]
  double dkx, dky;        // 2 pi / (n d)
  int nx, ny, ninst, rows, C;
};

constexpr int kRowMaxThreads = 256;
constexpr size_t kMaxSmemPerBlock = 227 * 1024;  // opt-in dynamic shared memory per block on GB300
constexpr int kColMaxThreads = 512;

// Shared-memory element counts (host and device use the same formulas).
// One padding slot per 128-byte line keeps strided Stockham writes free of
// bank conflicts.
__host__ __device__ constexpr int pad_shift(int elem_bytes) { return elem_bytes == 8 ? 4 : 3; }
__host__ __device__ constexpr int row_pad_n(int n, int elem_bytes) { return n + (n >> pad_shift(elem_bytes)); }
__host__ __device__ constexpr int row_stride(int n, int elem_bytes) { return 2 * row_pad_n(n, elem_bytes) + 2; }
__host__ __device__ constexpr int col_smem_elems(int n, int c, int elem_bytes) {
  return n * c + ((n * c) >> pad_shift(elem_bytes)) + 1;
}

// log2 of the values each thread holds in the block FFTs (one component per
// thread).  Row pass: 16 complex64 or 8 complex128, 16 complex128 at 4096 so
// that one row fits a 512-thread block.  Column pass: the same, with 16
// complex128 from 2048 up.  Energy row pass (two components per thread):
// 16 complex64, 8 complex128.
__host__ __device__ constexpr int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int row_loge_for(int logn, int es) {
  return es == 8 ? imin(logn, 4) : (logn >= 12 ? 4 : imin(logn, 3));
}
__host__ __device__ constexpr int col_loge_for(int logn, int es) {
  return es == 8 ? imin(logn, 4) : (logn >= 11 ? 4 : imin(logn, 3));
}
__host__ __device__ constexpr int erow_loge_for(int logn, int es) { return imin(logn, es == 8 ? 4 : 3); }

// Launch geometry of the fused passes (host and device agree on it).
struct LaunchShape {
  int elems_per_thread;   // E: elements of one sequence held per thread
  int threads;            // block size
  int blocks_x;           // blocks per instance (row groups or column groups)
  int rows_or_cols;       // rows per block (row pass) or columns per block (column pass)
  size_t smem;            // dynamic shared memory bytes
};

// Per-precision launchers (T = float for SPGPE_C64, double for SPGPE_C128),
// explicitly instantiated in kernels_row.cu and kernels_col.cu.  They return
// cudaGetLastError() after the launch.
template <class T> LaunchShape row_shape(int nx, int ny);
// The row pass of one flag combination (plain / persistent), instantiated per
// flag group in the kernels_row_*.cu units; launch_row / launch_row_p
// dispatch on the flags (kernels_row_dispatch.cu).
template <class T, int F> cudaError_t launch_row_f(RowArgs a, cudaStream_t s);
template <class T, int F> cudaError_t launch_row_pf(RowArgs a, cudaStream_t s, int sms);
template <class T> LaunchShape col_shape(int nx, int ny);
template <class T> cudaError_t launch_row(int flags, RowArgs a, cudaStream_t s);
template <class T> cudaError_t launch_col(bool imag, ColArgs a, cudaStream_t s);
template <class T> cudaError_t launch_energy(EnergyArgs a, cudaStream_t s, int *row_blocks, int *col_blocks);
template <class T> cudaError_t launch_norm(const void *psi, long plane, int ninst, double *partials, int blocks,
                                           cudaStream_t s);
template <class T> cudaError_t launch_residual(const void *psi, const void *prev, long plane, int ninst,
                                               double *partials, int blocks, cudaStream_t s);
template <class T> cudaError_t launch_ref_R(bool imag, const RowArgs &a, cudaStream_t s);
// Persistent passes (async tile loads; psi must be 16-byte aligned).  sms is
// the device's multiprocessor count.  They return cudaErrorNotSupported for
// shapes they do not cover (the caller then runs the plain pass).  The
// column pass reads psi through `map`,
// a 2D tensor map over [ninst*2*ny rows][nx complex] with a box of
// colp_cols<T>() columns by min(ny, 256) rows.
template <class T> cudaError_t launch_row_p(int flags, RowArgs a, cudaStream_t s, int sms);
template <class T> int colp_cols(int nx, int ny);
template <class T> cudaError_t launch_col_p(bool imag, ColArgs a, const CUtensorMap &map, cudaStream_t s, int sms);
template <class T> cudaError_t launch_ref_K(const ColArgs &a, cudaStream_t s);
// Warp-local column pass (complex64, ny = 256, nx >= 16; otherwise
// cudaErrorNotSupported): psi through `map`, a tensor map like the one above
// but with 16 x 256 boxes and the 128-byte swizzle.
template <class T> cudaError_t launch_col_w(bool imag, ColArgs a, const CUtensorMap &map, cudaStream_t s, int sms);
// Geometry of the Sec. 6 observables: grid, radial bin width h and count nb.
struct ObsGeom {
  int nx, ny, nb;
  double xmax, ymax, dx, dy, h;
};
// phase 0: FP64 sums {rho_up rho_dn, rho_up^2, rho_dn^2, rho_up + rho_dn} per
// block and instance into partials ([ninst][sum_blocks][4]) and the radial
// histogram of the total density into hist ([ninst][nb], zeroed by the
// caller); phase 1: winding numbers around radius R[inst] with npts points
// into wind ([ninst][2]).  es = bytes per complex element.
cudaError_t launch_observables(int es, const void *psi, const ObsGeom &g, int ninst, double *partials,
                               int sum_blocks, double *hist, const double *R, int npts, double *wind, int phase,
                               cudaStream_t st);
// psi += sigma xi over ninst instances of n2 = 2 nx ny elements (global index
// of the first: inst0), from the counter-based SplitMix64 stream `seed`.
cudaError_t launch_add_noise(int es, void *psi, long n2, int ninst, long inst0, double sigma, unsigned long long seed,
                             int sms, cudaStream_t st);

// Round complex128 to complex64 (src_es 16, dst_es 8) or widen complex64 to
// complex128 (8, 16): n complex values, grid of at most 8 blocks per SM.
cudaError_t launch_convert(const void *src, int src_es, void *dst, int dst_es, long n, int sms, cudaStream_t s);

}  // namespace spgpe
