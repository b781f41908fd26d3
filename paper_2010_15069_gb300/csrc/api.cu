// C ABI of the fused TSSP solver (include/spgpe.h): context, operator tables,
// step scheduling, reductions, and the cuFFT comparator.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cufft.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "spgpe.h"
#include "async_copy.cuh"
#include "internal.h"
#include "twiddles.h"

namespace spgpe {
// The bounded-wait failure probe (kernels_misc.cu).
cudaError_t launch_wait_probe(int *flags, long long budget, cudaStream_t s);
}  // namespace spgpe

using namespace spgpe;

namespace {

const double kTwoPi = 6.28318530717958647692528676655900577;

thread_local std::string g_init_error;

bool pow2_in_range(int n) { return n >= 8 && n <= 4096 && (n & (n - 1)) == 0; }

constexpr int kResidualBlocks = 128;  // blocks per instance of the residual reduction

}  // namespace

struct spgpe_ctx {
  int nx = 0, ny = 0, ninst = 1, dtype = 0;
  double xmax = 0, ymax = 0, dx = 0, dy = 0;
  cudaStream_t st = nullptr;
  size_t es = 0;  // bytes per complex element

  // Host FP64 model, per instance: x pieces [ninst][nx][3] = (V, delta, Omega),
  // y pieces [ninst][ny][3], couplings [ninst][4] = (g11, g22, g12, kL).
  std::vector<double> hx, hy, hg;
  std::vector<char> inst_set;
  bool has2d = false;

  // Device tables.
  void *d_twx = nullptr, *d_twy = nullptr;  // twiddle tables: row plan (x), column plan (y)
  void *d_twe = nullptr;                     // energy-row plan (x), when it differs from the row plan
  void *d_tabx = nullptr, *d_taby = nullptr;  // step tables for (tab_dt, tab_imag)
  void *d_rawx = nullptr, *d_rawy = nullptr;  // raw (V, delta, Omega) for energies
  void *d_pot2d = nullptr;
  void *d_kxt = nullptr, *d_kyt = nullptr;
  double *d_gpar = nullptr;
  double *d_partials = nullptr;
  size_t n_partials = 0;
  unsigned *d_counters = nullptr;
  double *d_scale = nullptr;
  double *d_scale2 = nullptr;  // second scale buffer of the lagged renormalisation
  void *d_scale_t = nullptr;   // both scale buffers in the working precision, [2][ninst][2]
  void *d_cfac = nullptr;      // [ninst][2] working precision: the lagged column pass's correction
  int *d_flags = nullptr;
  int *d_active = nullptr;    // [ninst] per-instance step mask (relaxation freezes converged instances)
  bool use_active = false;
  void *d_scratch = nullptr;  // psi-sized: energy transform / residual previous state
  void *d_stage = nullptr;    // psi-sized: staging of host spinors
  double *d_obs = nullptr;    // observables: radial histogram, radii, windings
  size_t n_obs = 0;
  double tab_dt = NAN;
  int tab_imag = -1;
  int omega_pieces = 0;
  double vbound2d = 0.0;  // max |V +- delta/2| of the 2D arrays (0 when separable)
  std::vector<double> h2d;  // host copy of the 2D {V + delta/2, V - delta/2, Omega, 0} table
  unsigned model_version = 0;

  // Precision ladder (spgpe_relax): a complex64 twin of a complex128 context
  // with the same model, and its spinor buffer.
  spgpe_ctx *twin = nullptr;
  unsigned twin_version = ~0u;
  void *d_psi64 = nullptr;

  cufftHandle plan = 0;
  bool plan_ok = false;

  // Persistent passes: multiprocessor count, and the column tensor map of the
  // spinor buffer last stepped (rebuilt when the buffer changes).
  int sms = 0;
  bool persistent_row = true;
  bool persistent_col = true;
  bool warp_col = true;  // the warp-local column pass where it applies (ny = 256, complex64)
  int host_chunks = 8;   // chunks of instances a host batch goes through (copies overlap steps)
  const void *map_psi = nullptr, *map_sw_psi = nullptr;
  int map_ninst = 0, map_sw_ninst = 0;
  CUtensorMap map{}, map_sw{};
  // Host spinors of a batch go through in chunks of instances: copies in on
  // cp_in, the steps on st, copies out on cp_out (streams and events created
  // on first use).
  cudaStream_t cp_in = nullptr, cp_out = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_done;
  void *d_gparT = nullptr;

  // Batch over several grid sizes: the size classes are child contexts, each
  // on a stream of its own; this context only dispatches to them.  Class k
  // holds global instances cls_first[k] .. cls_first[k] + ninst_k - 1 at byte
  // offset cls_off[k] of the spinor buffer.
  std::vector<spgpe_ctx *> cls;
  std::vector<int> cls_first;
  std::vector<size_t> cls_off;
  size_t multi_bytes = 0;
  cudaEvent_t fork_ev = nullptr;  // parent: recorded on its stream before the classes start
  cudaEvent_t join_ev = nullptr;  // child: recorded on its stream when its work is queued
  bool own_stream = false;        // child: the stream was created by the library

  std::string err;
  int last_launches = 0;

  // Optional per-launch timing (spgpe_set_timing): event pairs per kind.
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;

  size_t psi_bytes() const { return cls.empty() ? (size_t)ninst * 2 * nx * ny * es : multi_bytes; }
  long plane() const { return (long)nx * ny; }
};

namespace {

int fail(spgpe_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  else g_init_error = msg;
  return code;
}

int cuda_fail(spgpe_ctx *c, cudaError_t e, const char *what) {
  return fail(c, SPGPE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(ctx, expr)                                   \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #expr); \
  } while (0)

bool all_finite(const double *p, size_t n) {
  if (!p) return true;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Upload FP64 values as the working precision T (float or double).
int upload(spgpe_ctx *c, void *dst, const std::vector<double> &src) {
  if (c->dtype == SPGPE_C64) {
    std::vector<float> f(src.begin(), src.end());
    CK(c, cudaMemcpyAsync(dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice, c->st));
  } else {
    CK(c, cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
  }
  return SPGPE_OK;
}

int dev_alloc(spgpe_ctx *c, void **p, size_t bytes) {
  if (*p) return SPGPE_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? SPGPE_ENOMEM : SPGPE_ECUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return SPGPE_OK;
}

void free_all(spgpe_ctx *c) {
  if (c->d_gparT) cudaFree(c->d_gparT);
  for (auto &u : c->ev_used) {
    cudaEventDestroy(u.second.first);
    cudaEventDestroy(u.second.second);
  }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  void *ps[] = {c->d_twx, c->d_twy, c->d_twe, c->d_tabx, c->d_taby, c->d_rawx, c->d_rawy, c->d_pot2d, c->d_kxt,
                c->d_kyt, c->d_gpar, c->d_partials, c->d_counters, c->d_scale, c->d_scale2, c->d_scale_t,
                c->d_cfac, c->d_flags, c->d_active, c->d_scratch, c->d_stage};
  for (void *p : ps)
    if (p) cudaFree(p);
  if (c->plan_ok) cufftDestroy(c->plan);
  if (c->d_psi64) cudaFree(c->d_psi64);
  if (c->d_obs) cudaFree(c->d_obs);
  if (c->twin) {
    free_all(c->twin);
    delete c->twin;
  }
  for (spgpe_ctx *k : c->cls) {
    cudaStreamSynchronize(k->st);
    free_all(k);
    delete k;
  }
  for (cudaEvent_t e : c->ev_in) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_done) cudaEventDestroy(e);
  if (c->cp_in) cudaStreamDestroy(c->cp_in);
  if (c->cp_out) cudaStreamDestroy(c->cp_out);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
}

int log2i(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

double kval(int i, int n, double d) { return kTwoPi * (i < n / 2 ? i : i - n) / (n * d); }

// Raw (V, delta, Omega, 0) tables for the energy kernels.
int upload_raw(spgpe_ctx *c) {
  std::vector<double> rx((size_t)c->ninst * c->nx * 4), ry((size_t)c->ninst * c->ny * 4);
  for (int i = 0; i < c->ninst; ++i) {
    for (int x = 0; x < c->nx; ++x)
      for (int k = 0; k < 3; ++k) rx[((size_t)i * c->nx + x) * 4 + k] = c->hx[((size_t)i * c->nx + x) * 3 + k];
    for (int y = 0; y < c->ny; ++y)
      for (int k = 0; k < 3; ++k) ry[((size_t)i * c->ny + y) * 4 + k] = c->hy[((size_t)i * c->ny + y) * 3 + k];
  }
  int r = upload(c, c->d_rawx, rx);
  if (r) return r;
  r = upload(c, c->d_rawy, ry);
  if (r) return r;
  CK(c, cudaMemcpyAsync(c->d_gpar, c->hg.data(), c->hg.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
  // Working-precision couplings {g11, g22, g12, Vb}, Vb = max |V +- delta/2| of
  // the instance: the kernels bound the D phase with it to pick the small-phase
  // series for a whole warp.
  std::vector<double> gt(c->hg.size());
  for (int i = 0; i < c->ninst; ++i) {
    double vb = 0.0;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
      for (int x = 0; x < c->nx; ++x) {
        const double *h = &c->hx[((size_t)i * c->nx + x) * 3];
        const double v = h[0] + 0.5 * sgn * h[1];
        xmin = std::min(xmin, v);
        xmax = std::max(xmax, v);
      }
      for (int y = 0; y < c->ny; ++y) {
        const double *h = &c->hy[((size_t)i * c->ny + y) * 3];
        const double v = h[0] + 0.5 * sgn * h[1];
        ymin = std::min(ymin, v);
        ymax = std::max(ymax, v);
      }
      vb = std::max(vb, std::max(std::fabs(xmin + ymin), std::fabs(xmax + ymax)));
    }
    gt[4 * i] = c->hg[4 * i];
    gt[4 * i + 1] = c->hg[4 * i + 1];
    gt[4 * i + 2] = c->hg[4 * i + 2];
    gt[4 * i + 3] = vb + c->vbound2d;
  }
  if ((r = upload(c, c->d_gparT, gt))) return r;
  c->tab_dt = NAN;  // step tables depend on the model
  return SPGPE_OK;
}

// Step tables for substep dt (real or imaginary time):
//   x/y step tables {p(V + delta/2), p(V - delta/2), X constants} of the
//   separable pieces: p(v) = -(dt/4) v, the half phase of D(dt/2), in real
//   time; p(v) = exp(-(dt/2) v), the potential factors of D(dt/2), which
//   multiply to the factor of the sum, in imaginary time.  X constants for
//   the angle a = Omega_piece dt / 8 of X(dt/4), each applied as three shears:
//   (tan(a/2), sin a) of the rotation in real time, (tanh(a/2), sinh a) of
//   the hyperbolic rotation in imaginary time;
//   K tables a_j(kx) - 1 with a_j = exp(-i dt (kx^2/2 -+ kL kx)) and b(ky) - 1
//   with b = exp(-i dt ky^2/2) (imaginary time: exp(-dt (...)) - 1); the
//   1/(nx ny) of the inverse transform is applied in the kernel.
int ensure_tables(spgpe_ctx *c, double dt, int imag) {
  if (c->tab_dt == dt && c->tab_imag == imag) return SPGPE_OK;
  const int nx = c->nx, ny = c->ny, ni = c->ninst;
  std::vector<double> tx((size_t)ni * nx * 4), ty((size_t)ni * ny * 4);
  bool too_big = false;
  auto rot = [&](double ang, double &mm, double &ss) {
    if (imag) {
      mm = std::tanh(0.5 * ang);
      ss = std::sinh(ang);
    } else {
      if (std::fabs(ang) > 0.25 * kTwoPi) too_big = true;
      mm = std::tan(0.5 * ang);
      ss = std::sin(ang);
    }
  };
  // exp(-i th) - 1 (real time) or exp(-th) - 1 (imaginary time)
  auto em1 = [&](double th, double *o) {
    if (imag) {
      o[0] = std::expm1(-th);
      o[1] = 0.0;
    } else {
      const double sh = std::sin(0.5 * th);
      o[0] = -2.0 * sh * sh;
      o[1] = -std::sin(th);
    }
  };
  // potential entries: htau (V +- delta/2) with htau = -dt/4, the half phase
  // of D(dt/2) (real time), or the factors exp(-(dt/2) (V +- delta/2)) of
  // D(dt/2) in imaginary time
  auto pot = [&](double v) { return imag ? std::exp(-0.5 * dt * v) : -0.25 * dt * v; };
  for (int i = 0; i < ni; ++i) {
    for (int x = 0; x < nx; ++x) {
      const double *h = &c->hx[((size_t)i * nx + x) * 3];
      double *o = &tx[((size_t)i * nx + x) * 4];
      o[0] = pot(h[0] + 0.5 * h[1]);
      o[1] = pot(h[0] - 0.5 * h[1]);
      rot(h[2] * dt / 8.0, o[2], o[3]);
    }
    for (int y = 0; y < ny; ++y) {
      const double *h = &c->hy[((size_t)i * ny + y) * 3];
      double *o = &ty[((size_t)i * ny + y) * 4];
      o[0] = pot(h[0] + 0.5 * h[1]);
      o[1] = pot(h[0] - 0.5 * h[1]);
      rot(h[2] * dt / 8.0, o[2], o[3]);
    }
  }
  std::vector<double> kx((size_t)ni * 2 * nx * 2), ky((size_t)ny * 2);
  for (int i = 0; i < ni; ++i) {
    const double kL = c->hg[4 * i + 3];
    for (int j = 0; j < 2; ++j)
      for (int x = 0; x < nx; ++x) {
        const double k = kval(x, nx, c->dx);
        em1(dt * (0.5 * k * k + (j == 0 ? -kL : kL) * k), &kx[(((size_t)i * 2 + j) * nx + x) * 2]);
      }
  }
  for (int y = 0; y < ny; ++y) {
    const double k = kval(y, ny, c->dy);
    em1(dt * 0.5 * k * k, &ky[2 * (size_t)y]);
  }
  if (too_big) return fail(c, SPGPE_EINVAL, "|Omega| dt / 8 exceeds pi/2: time step too large for the Raman coupling");
  c->omega_pieces = 0;
  for (int i = 0; i < ni; ++i) {
    for (int y = 0; y < ny; ++y)
      if (c->hy[((size_t)i * ny + y) * 3 + 2] != 0.0) c->omega_pieces |= 1;
    for (int x = 0; x < nx; ++x)
      if (c->hx[((size_t)i * nx + x) * 3 + 2] != 0.0) c->omega_pieces |= 2;
  }
  int r;
  if ((r = upload(c, c->d_tabx, tx)) || (r = upload(c, c->d_taby, ty)) || (r = upload(c, c->d_kxt, kx)) ||
      (r = upload(c, c->d_kyt, ky)))
    return r;
  c->tab_dt = dt;
  c->tab_imag = imag;
  return SPGPE_OK;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

RowArgs row_args(spgpe_ctx *c, void *psi, double dt) {
  RowArgs a{};
  a.psi = psi;
  a.tabx = c->d_tabx;
  a.taby = c->d_taby;
  a.pot2d = c->has2d ? c->d_pot2d : nullptr;
  a.tw = c->d_twx;
  a.gpar = c->d_gpar;
  a.gparT = c->d_gparT;
  a.tau = 0.5 * dt;
  a.xang = dt / 8.0;
  a.htau_d = c->tab_imag ? -a.tau : -0.5 * a.tau;
  a.htau_f = (float)a.htau_d;
  a.xang_f = (float)a.xang;
  a.omega_pieces = c->omega_pieces;
  a.partials = c->d_partials;
  a.counters = c->d_counters;
  a.scale = c->d_scale;
  a.scale_t = c->d_scale_t;
  a.scale_pred = c->d_scale2;
  a.scale_pred_t = static_cast<char *>(c->d_scale_t) + (size_t)c->ninst * 2 * (c->es / 2);
  a.cfac = nullptr;
  a.tgt0 = 0.5;
  a.tgt1 = 0.5;
  a.norm_mode = 0;
  a.wgt = c->dx * c->dy;
  a.active = c->use_active ? c->d_active : nullptr;
  a.flags = c->d_flags;
  a.nx = c->nx;
  a.ny = c->ny;
  a.ninst = c->ninst;
  return a;
}

// The same arguments for instances i0 .. i0 + ni - 1 only: psi and every
// per-instance table seen from instance i0 (the kernels index instances
// from zero); psi is the batch's base pointer.
template <class P> P *skip(P *p, size_t bytes) {
  return p ? reinterpret_cast<P *>(reinterpret_cast<unsigned char *>(const_cast<void *>(static_cast<const void *>(p))) +
                                   bytes)
           : p;
}

void restrict_row(const spgpe_ctx *c, RowArgs &a, int i0, int ni) {
  const size_t es = c->es, i = (size_t)i0;
  a.psi = skip(a.psi, i * 2 * c->plane() * es);
  a.tabx = skip(a.tabx, i * c->nx * 2 * es);
  a.taby = skip(a.taby, i * c->ny * 2 * es);
  a.gpar = skip(a.gpar, i * 4 * sizeof(double));
  a.gparT = skip(a.gparT, i * 4 * (es / 2));
  a.partials = skip(a.partials, i * c->ny * 2 * sizeof(double));
  a.counters = skip(a.counters, i * sizeof(unsigned));
  a.scale = skip(a.scale, i * 2 * sizeof(double));
  a.scale_pred = skip(a.scale_pred, i * 2 * sizeof(double));
  a.scale_t = skip(a.scale_t, i * 2 * (es / 2));
  a.scale_pred_t = skip(a.scale_pred_t, i * 2 * (es / 2));
  a.cfac = skip(a.cfac, i * 2 * (es / 2));
  a.active = skip(a.active, i * sizeof(int));
  a.ninst = ni;
}

void restrict_col(const spgpe_ctx *c, ColArgs &a, int i0, int ni) {
  const size_t es = c->es, i = (size_t)i0;
  a.psi = skip(a.psi, i * 2 * c->plane() * es);
  a.kxt = skip(a.kxt, i * 2 * c->nx * es);
  a.cfac = skip(a.cfac, i * 2 * (es / 2));
  a.active = skip(a.active, i * sizeof(int));
  a.ninst = ni;
}

ColArgs col_args(spgpe_ctx *c, void *psi) {
  ColArgs a{};
  a.psi = psi;
  a.kxt = c->d_kxt;
  a.kyt = c->d_kyt;
  a.tw = c->d_twy;
  a.inv_d = 1.0 / ((double)c->nx * c->ny);
  a.inv_f = (float)a.inv_d;
  a.flags = c->d_flags;
  a.active = c->use_active ? c->d_active : nullptr;
  a.nx = c->nx;
  a.ny = c->ny;
  a.ninst = c->ninst;
  return a;
}

cudaEvent_t take_event(spgpe_ctx *c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int kind_of_row(int flags) {
  switch (flags) {
    case kRealFirst: return 0;
    case kRealMid: return 1;
    case kRealLast: return 2;
    case kImagFirst: return 4;
    case kImagB: return 5;
    case kImagA: return 6;
    case kImagLag: return 9;
    default: return 7;
  }
}

template <class F> cudaError_t timed(spgpe_ctx *c, int kind, F &&launch) {
  ++c->last_launches;
  if (!c->timing) return launch();
  cudaEvent_t a = take_event(c), b = take_event(c);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaEventRecord(a, c->st);
  if (e != cudaSuccess) return e;
  e = launch();
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(b, c->st);
  c->ev_used.push_back({kind, {a, b}});
  return e;
}

bool aligned16(const void *psi) { return (reinterpret_cast<uintptr_t>(psi) & 15) == 0; }

cudaError_t row(spgpe_ctx *c, int flags, const RowArgs &a) {
  const bool p = c->persistent_row && c->sms > 0 && aligned16(a.psi);
  return timed(c, kind_of_row(flags), [&] {
    if (p) {
      const cudaError_t e = c->dtype == SPGPE_C64 ? launch_row_p<float>(flags, a, c->st, c->sms)
                                                  : launch_row_p<double>(flags, a, c->st, c->sms);
      if (e != cudaErrorNotSupported) return e;
    }
    return c->dtype == SPGPE_C64 ? launch_row<float>(flags, a, c->st) : launch_row<double>(flags, a, c->st);
  });
}

// Tensor maps over the spinor buffer viewed as [ninst*2*ny rows][nx complex]
// (8-byte elements: one complex64, or half a complex128): `map` with boxes
// of C complex columns by min(ny, 256) rows for the persistent column pass,
// `map_sw` with 16 x 256 boxes and the 128-byte swizzle for the warp-local one.
cudaError_t encode_map(spgpe_ctx *c, const void *psi, int ninst, CUtensorMap *m, int cols, bool swizzle) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int xm = c->dtype == SPGPE_C64 ? 1 : 2;
  const cuuint64_t dims[2] = {(cuuint64_t)c->nx * xm, (cuuint64_t)ninst * 2 * c->ny};
  const cuuint64_t strides[1] = {(cuuint64_t)c->nx * c->es};
  const cuuint32_t box[2] = {(cuuint32_t)(cols * xm), (cuuint32_t)std::min(c->ny, 256)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(m, c->dtype == SPGPE_C64 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                            const_cast<void *>(psi), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t ensure_map(spgpe_ctx *c, const void *psi, int ninst) {
  if (c->map_psi == psi && c->map_ninst == ninst) return cudaSuccess;
  const int C = c->dtype == SPGPE_C64 ? colp_cols<float>(c->nx, c->ny) : colp_cols<double>(c->nx, c->ny);
  const cudaError_t e = encode_map(c, psi, ninst, &c->map, C, false);
  if (e == cudaSuccess) {
    c->map_psi = psi;
    c->map_ninst = ninst;
  }
  return e;
}

cudaError_t ensure_map_sw(spgpe_ctx *c, const void *psi, int ninst) {
  if (c->map_sw_psi == psi && c->map_sw_ninst == ninst) return cudaSuccess;
  const cudaError_t e = encode_map(c, psi, ninst, &c->map_sw, 16, true);
  if (e == cudaSuccess) {
    c->map_sw_psi = psi;
    c->map_sw_ninst = ninst;
  }
  return e;
}

bool warp_col_applies(const spgpe_ctx *c) { return c->dtype == SPGPE_C64 && c->ny == 256 && c->nx >= 16; }

cudaError_t col(spgpe_ctx *c, bool imag, const ColArgs &a) {
  const bool ok16 = c->sms > 0 && aligned16(a.psi);
  bool w = c->warp_col && ok16 && warp_col_applies(c);
  if (w && ensure_map_sw(c, a.psi, a.ninst) != cudaSuccess) w = false;
  bool p = !w && c->persistent_col && ok16;
  if (p && ensure_map(c, a.psi, a.ninst) != cudaSuccess) p = false;
  return timed(c, imag ? 8 : 3, [&] {
    if (w) {
      const cudaError_t e = launch_col_w<float>(imag, a, c->map_sw, c->st, c->sms);
      if (e != cudaErrorNotSupported) return e;
    }
    if (p) {
      const cudaError_t e = c->dtype == SPGPE_C64 ? launch_col_p<float>(imag, a, c->map, c->st, c->sms)
                                                  : launch_col_p<double>(imag, a, c->map, c->st, c->sms);
      if (e != cudaErrorNotSupported) return e;
    }
    return c->dtype == SPGPE_C64 ? launch_col<float>(imag, a, c->st) : launch_col<double>(imag, a, c->st);
  });
}

int check_ready(spgpe_ctx *c) {
  if (!c) return SPGPE_EINVAL;
  for (spgpe_ctx *k : c->cls)
    if (check_ready(k)) return fail(c, SPGPE_ESTATE, "potentials not set for every instance");
  for (char s : c->inst_set)
    if (!s) return fail(c, SPGPE_ESTATE, "potentials not set for every instance");
  return SPGPE_OK;
}

// Resolve a caller spinor: device pointers are used in place, host spinors are
// staged through the context's device buffer.
int begin_psi(spgpe_ctx *c, const void *psi, void **dev, bool *host) {
  *host = !is_device_ptr(psi);
  if (!*host) {
    *dev = const_cast<void *>(psi);
    return SPGPE_OK;
  }
  int r = dev_alloc(c, &c->d_stage, c->psi_bytes());
  if (r) return r;
  CK(c, cudaMemcpyAsync(c->d_stage, psi, c->psi_bytes(), cudaMemcpyHostToDevice, c->st));
  *dev = c->d_stage;
  return SPGPE_OK;
}

int end_psi(spgpe_ctx *c, void *psi, bool host) {
  if (!host) return SPGPE_OK;
  CK(c, cudaMemcpyAsync(psi, c->d_stage, c->psi_bytes(), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  return SPGPE_OK;
}

// Host spinor of a batch: copy in, step and copy out in chunks of instances,
// the copy in of a chunk (cp_in) and the copy out of the one before
// (cp_out) overlapping the steps of another (on st).  run(i0, ni, base)
// queues the steps of instances i0 .. i0 + ni - 1 of the staged batch at
// `base` on st.  Synchronises.
template <class F> int host_pipeline(spgpe_ctx *c, void *psi, F &&run) {
  const int nch = std::min(c->ninst, c->host_chunks);
  int r = dev_alloc(c, &c->d_stage, c->psi_bytes());
  if (r) return r;
  if (!c->cp_in) {
    CK(c, cudaStreamCreateWithFlags(&c->cp_in, cudaStreamNonBlocking));
    CK(c, cudaStreamCreateWithFlags(&c->cp_out, cudaStreamNonBlocking));
  }
  while ((int)c->ev_in.size() < nch + 1) {
    cudaEvent_t a = nullptr, b = nullptr;
    CK(c, cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    CK(c, cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    c->ev_in.push_back(a);
    c->ev_done.push_back(b);
  }
  const size_t per = 2 * (size_t)c->plane() * c->es;
  unsigned char *dev = static_cast<unsigned char *>(c->d_stage), *hst = static_cast<unsigned char *>(psi);
  auto queue = [&]() -> int {
    // the copies start after the work already queued on the context's stream
    CK(c, cudaEventRecord(c->ev_done[nch], c->st));
    CK(c, cudaStreamWaitEvent(c->cp_in, c->ev_done[nch], 0));
    for (int k = 0; k < nch; ++k) {
      const int i0 = (int)((long)k * c->ninst / nch), i1 = (int)((long)(k + 1) * c->ninst / nch);
      const size_t off = (size_t)i0 * per, bytes = (size_t)(i1 - i0) * per;
      CK(c, cudaMemcpyAsync(dev + off, hst + off, bytes, cudaMemcpyHostToDevice, c->cp_in));
      CK(c, cudaEventRecord(c->ev_in[k], c->cp_in));
      CK(c, cudaStreamWaitEvent(c->st, c->ev_in[k], 0));
      int rr = run(i0, i1 - i0, c->d_stage);
      if (rr) return rr;
      CK(c, cudaEventRecord(c->ev_done[k], c->st));
      CK(c, cudaStreamWaitEvent(c->cp_out, c->ev_done[k], 0));
      CK(c, cudaMemcpyAsync(hst + off, dev + off, bytes, cudaMemcpyDeviceToHost, c->cp_out));
    }
    return SPGPE_OK;
  };
  if ((r = queue())) {
    // copies already queued still use the caller's buffer: let them finish
    cudaStreamSynchronize(c->cp_in);
    cudaStreamSynchronize(c->cp_out);
    cudaStreamSynchronize(c->st);
    cudaGetLastError();
    return r;
  }
  CK(c, cudaStreamSynchronize(c->cp_out));
  CK(c, cudaStreamSynchronize(c->st));
  return SPGPE_OK;
}

int read_flags(spgpe_ctx *c) {
  int h = 0;
  CK(c, cudaMemcpyAsync(&h, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  if (h) {
    CK(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->st));
    if (h & kErrBounds)
      return fail(c, SPGPE_EBOUNDS, "an index fell outside its buffer (bounds-checked build; the access was skipped)");
    if (h & kErrTimeout) return fail(c, SPGPE_ETIMEOUT, "a tile transfer did not complete within the wait limit");
    return fail(c, SPGPE_ENONFINITE, "non-finite or zero atom number met during imaginary-time renormalisation");
  }
  return SPGPE_OK;
}

int init_common(spgpe_ctx **out, int nx, int ny, double xmax, double ymax, int ninst, int dtype, void *stream) {
  if (!out) return fail(nullptr, SPGPE_EINVAL, "out is NULL");
  *out = nullptr;
  if (!pow2_in_range(nx) || !pow2_in_range(ny))
    return fail(nullptr, SPGPE_EINVAL, "nx and ny must be powers of two in [8, 4096]");
  if (!(std::isfinite(xmax) && xmax > 0 && std::isfinite(ymax) && ymax > 0))
    return fail(nullptr, SPGPE_EINVAL, "xmax and ymax must be finite and positive");
  if (dtype != SPGPE_C64 && dtype != SPGPE_C128) return fail(nullptr, SPGPE_EINVAL, "dtype must be SPGPE_C64 or SPGPE_C128");
  if (ninst < 1 || ninst > 65535) return fail(nullptr, SPGPE_EINVAL, "ninst must be in [1, 65535]");
  spgpe_ctx *c = new (std::nothrow) spgpe_ctx();
  if (!c) return fail(nullptr, SPGPE_ENOMEM, "host allocation failed");
  c->nx = nx;
  c->ny = ny;
  c->ninst = ninst;
  c->dtype = dtype;
  c->xmax = xmax;
  c->ymax = ymax;
  c->dx = 2.0 * xmax / nx;
  c->dy = 2.0 * ymax / ny;
  c->st = reinterpret_cast<cudaStream_t>(stream);
  c->es = dtype == SPGPE_C64 ? 8 : 16;
  c->hx.assign((size_t)ninst * nx * 3, 0.0);
  c->hy.assign((size_t)ninst * ny * 3, 0.0);
  c->hg.assign((size_t)ninst * 4, 0.0);
  c->inst_set.assign(ninst, 0);
  const size_t es = c->es, q = 2 * es;
  // partial sums: row-pass renormalisation (ny blocks at most), energies
  // (6 per row block + 2 per column block), norms (256 blocks of 2)
  c->n_partials = (size_t)ninst * (6 * (size_t)ny + 2 * (size_t)nx + 2 * 1024);
  int r;
  if ((r = dev_alloc(c, &c->d_tabx, (size_t)ninst * nx * q)) || (r = dev_alloc(c, &c->d_taby, (size_t)ninst * ny * q)) ||
      (r = dev_alloc(c, &c->d_rawx, (size_t)ninst * nx * q)) || (r = dev_alloc(c, &c->d_rawy, (size_t)ninst * ny * q)) ||
      (r = dev_alloc(c, &c->d_kxt, (size_t)ninst * 2 * nx * es)) || (r = dev_alloc(c, &c->d_kyt, ny * es)) ||
      (r = dev_alloc(c, (void **)&c->d_gpar, (size_t)ninst * 4 * sizeof(double))) ||
      (r = dev_alloc(c, &c->d_gparT, (size_t)ninst * 4 * sizeof(double))) ||
      (r = dev_alloc(c, (void **)&c->d_partials, c->n_partials * sizeof(double))) ||
      (r = dev_alloc(c, (void **)&c->d_counters, (size_t)ninst * sizeof(unsigned))) ||
      (r = dev_alloc(c, (void **)&c->d_scale, (size_t)ninst * 2 * sizeof(double))) ||
      (r = dev_alloc(c, (void **)&c->d_scale2, (size_t)ninst * 2 * sizeof(double))) ||
      (r = dev_alloc(c, &c->d_scale_t, (size_t)2 * ninst * 2 * sizeof(double))) ||
      (r = dev_alloc(c, &c->d_cfac, (size_t)ninst * 2 * sizeof(double))) ||
      (r = dev_alloc(c, (void **)&c->d_flags, sizeof(int))) ||
      (r = dev_alloc(c, (void **)&c->d_active, (size_t)ninst * sizeof(int)))) {
    g_init_error = c->err;
    free_all(c);
    delete c;
    return r;
  }
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->d_counters, 0, (size_t)ninst * sizeof(unsigned), c->st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->st)) != cudaSuccess) {
    g_init_error = cudaGetErrorString(e);
    free_all(c);
    delete c;
    return SPGPE_ECUDA;
  }
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      c->sms = 0;
    cudaGetLastError();
    // SPGPE_PERSISTENT selects the pass variants: 0 plain passes, 1 persistent
    // column passes only, 2 persistent row and column passes (default; the
    // column pass warp-local where it applies).  SPGPE_COLPASS=tma or warp
    // picks between the two persistent column passes.  spgpe_autotune
    // overrides both.
    const char *env = std::getenv("SPGPE_PERSISTENT");
    if (env && env[0] >= '0' && env[0] <= '2') {
      c->persistent_col = env[0] != '0';
      c->persistent_row = env[0] == '2';
      c->warp_col = env[0] != '0';
    }
    const char *cp = std::getenv("SPGPE_COLPASS");
    if (cp && std::strcmp(cp, "warp") == 0) c->warp_col = true;
    if (cp && std::strcmp(cp, "tma") == 0) c->warp_col = false;
    // SPGPE_HOST_CHUNKS: chunks of a host batch (1..64; default 8)
    const char *hc = std::getenv("SPGPE_HOST_CHUNKS");
    if (hc) {
      const int v = std::atoi(hc);
      if (v >= 1 && v <= 64) c->host_chunks = v;
    }
  }
  {
    const int lx = log2i(nx), ly = log2i(ny), esz = (int)es;
    const bool single = dtype == SPGPE_C64;
    const std::vector<double> wr = stage_twiddles(lx, row_loge_for(lx, esz), single);
    const std::vector<double> wc = stage_twiddles(ly, col_loge_for(ly, esz), single);
    const bool sep_e = erow_loge_for(lx, esz) != row_loge_for(lx, esz);
    const std::vector<double> we = sep_e ? stage_twiddles(lx, erow_loge_for(lx, esz), single) : std::vector<double>();
    auto put = [&](void **d, const std::vector<double> &w) -> int {
      int rr = dev_alloc(c, d, w.size() * (single ? sizeof(float) : sizeof(double)));
      return rr ? rr : upload(c, *d, w);
    };
    if (!(r = put(&c->d_twx, wr)) && !(r = put(&c->d_twy, wc)) && sep_e) r = put(&c->d_twe, we);
  }
  if (r) {
    g_init_error = c->err;
    free_all(c);
    delete c;
    return r;
  }
  *out = c;
  return SPGPE_OK;
}

// nsteps imaginary-time steps of a device spinor, all on the context's stream
// and without synchronising.  With `residual`, the last step also leaves the
// residual partials (||Psi_{n+1} - Psi_n||^2, ||Psi_n||^2 per block and
// instance) in d_partials for imag_collect.
//
// Step boundaries (the closing R(dt/2) of step s, the renormalisation, the
// opening R(dt/2) of step s + 1): exact, two row passes (kImagA ends the step
// and computes the scale, kImagB applies it and opens the next step); or,
// with `lagged`, for every boundary but the first and the one before a
// residual step, one row pass (kImagLag) that opens the next step on the
// spinor scaled by the previous boundary's scale, with the column pass after
// it multiplying by the exact scale over that prediction.  The two scale
// buffers alternate so that a pass never reads the buffer it writes.
int imag_enqueue(spgpe_ctx *c, void *p, double dtau, int nsteps, int norm_mode, double t0, double t1,
                 bool residual, int i0 = 0, int ni = -1, bool lagged = false) {
  int r;
  if ((r = ensure_tables(c, dtau, 1))) return r;
  if (residual && (r = dev_alloc(c, &c->d_scratch, c->psi_bytes()))) return r;
  RowArgs ra = row_args(c, p, dtau);
  ra.tgt0 = t0;
  ra.tgt1 = t1;
  ra.norm_mode = norm_mode;
  ra.cfac = c->d_cfac;
  ColArgs ca = col_args(c, p);
  if (ni >= 0) {  // a chunk of instances (host pipeline; no residual)
    restrict_row(c, ra, i0, ni);
    restrict_col(c, ca, i0, ni);
  }
  // the two scale buffers (FP64 and working precision) and the correction
  double *sc[2] = {ra.scale, const_cast<double *>(ra.scale_pred)};
  void *st[2] = {ra.scale_t, const_cast<void *>(ra.scale_pred_t)};
  void *cf = ra.cfac;
  ra.cfac = nullptr;
  // sc[last]: the buffer holding the most recent exact scale
  int last = 0;
  if (nsteps == 1 && residual) {
    // Psi_0 is the input itself
    CK(c, cudaMemcpyAsync(c->d_scratch, p, c->psi_bytes(), cudaMemcpyDeviceToDevice, c->st));
  }
  CK(c, row(c, kImagFirst, ra));
  CK(c, col(c, true, ca));
  for (int s = 1; s < nsteps; ++s) {
    const bool into_residual_step = residual && s == nsteps - 1;
    if (!lagged || s == 1 || into_residual_step) {
      ra.scale = sc[0];
      ra.scale_t = st[0];
      CK(c, row(c, kImagA, ra));
      last = 0;
      if (into_residual_step) {
        // keep Psi_n (normalised) for the residual of the last step
        CK(c, row(c, kImagScale, ra));
        CK(c, cudaMemcpyAsync(c->d_scratch, p, c->psi_bytes(), cudaMemcpyDeviceToDevice, c->st));
        CK(c, row(c, kImagFirst, ra));
      } else {
        CK(c, row(c, kImagB, ra));
      }
      CK(c, col(c, true, ca));
    } else {
      RowArgs rl = ra;
      rl.scale_pred = sc[last];
      rl.scale_pred_t = st[last];
      rl.scale = sc[last ^ 1];
      rl.scale_t = st[last ^ 1];
      rl.cfac = cf;
      CK(c, row(c, kImagLag, rl));
      ColArgs cl = ca;
      cl.cfac = cf;
      CK(c, col(c, true, cl));
      last ^= 1;
    }
  }
  ra.scale = sc[0];
  ra.scale_t = st[0];
  CK(c, row(c, kImagA, ra));
  CK(c, row(c, kImagScale, ra));
  if (residual) {
    ++c->last_launches;
    if (c->dtype == SPGPE_C64)
      CK(c, launch_residual<float>(p, c->d_scratch, c->plane(), c->ninst, c->d_partials, kResidualBlocks, c->st));
    else
      CK(c, launch_residual<double>(p, c->d_scratch, c->plane(), c->ninst, c->d_partials, kResidualBlocks, c->st));
  }
  return SPGPE_OK;
}

// Wait for the residual partials of imag_enqueue and reduce them on the host.
int imag_collect(spgpe_ctx *c, double dtau, double *residual_out) {
  std::vector<double> h((size_t)c->ninst * kResidualBlocks * 2);
  CK(c, cudaMemcpyAsync(h.data(), c->d_partials, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  for (int i = 0; i < c->ninst; ++i) {
    double num = 0, den = 0;
    for (int b = 0; b < kResidualBlocks; ++b) {
      num += h[((size_t)i * kResidualBlocks + b) * 2];
      den += h[((size_t)i * kResidualBlocks + b) * 2 + 1];
    }
    residual_out[i] = std::sqrt(num / den) / dtau;
  }
  return SPGPE_OK;
}

// Size classes of a multi-size batch: start them after the work already on
// the caller's stream, and make the caller's stream wait for what they queue.
int fork_classes(spgpe_ctx *c) {
  CK(c, cudaEventRecord(c->fork_ev, c->st));
  for (spgpe_ctx *k : c->cls) CK(c, cudaStreamWaitEvent(k->st, c->fork_ev, 0));
  return SPGPE_OK;
}

int join_classes(spgpe_ctx *c) {
  for (spgpe_ctx *k : c->cls) {
    CK(c, cudaEventRecord(k->join_ev, k->st));
    CK(c, cudaStreamWaitEvent(c->st, k->join_ev, 0));
  }
  return SPGPE_OK;
}

// A class's failure, reported by the batch.
int class_fail(spgpe_ctx *c, spgpe_ctx *k, int r) { return fail(c, r, k->err); }

// Class of a global instance index (-1 when out of range).
int class_of(const spgpe_ctx *c, int inst) {
  for (size_t k = 0; k < c->cls.size(); ++k)
    if (inst >= c->cls_first[k] && inst < c->cls_first[k] + c->cls[k]->ninst) return (int)k;
  return -1;
}

// Run `call(class, class spinor, first instance)` for every class of a
// multi-size batch between a fork and a join on the caller's stream; a host
// spinor is staged once for the whole batch.
template <class F> int for_classes(spgpe_ctx *c, const void *psi, bool write_back, F &&call) {
  void *p;
  bool host;
  int r = begin_psi(c, psi, &p, &host);
  if (r) return r;
  if ((r = fork_classes(c))) return r;
  int launches = 0;
  for (size_t k = 0; k < c->cls.size(); ++k) {
    r = call(c->cls[k], static_cast<char *>(p) + c->cls_off[k], c->cls_first[k]);
    launches += c->cls[k]->last_launches;
    if (r) return class_fail(c, c->cls[k], r);
  }
  if ((r = join_classes(c))) return r;
  c->last_launches = launches;
  if (host) {
    // a host spinor makes the call synchronous: report device-side errors now
    if (write_back) {
      if ((r = end_psi(c, const_cast<void *>(psi), true))) return r;
    } else {
      CK(c, cudaStreamSynchronize(c->st));
    }
    for (spgpe_ctx *k : c->cls)
      if ((r = read_flags(k))) return class_fail(c, k, r);
  }
  return SPGPE_OK;
}

// Host spinor of a multi-size batch: each class's instances go through in
// chunks as in host_pipeline, the copies on the batch's two copy streams and
// the steps on the class's own stream, so that the copies of one chunk
// overlap the steps of the chunks and classes queued before it.
// run(k, i0, ni, base) queues the steps of instances i0 .. i0 + ni - 1 of
// class k (in the class's own numbering) of the class spinor at `base` on the
// class's stream.  Synchronises; sums the classes' launch counts.
template <class F> int host_pipeline_multi(spgpe_ctx *c, void *psi, F &&run) {
  int r = dev_alloc(c, &c->d_stage, c->psi_bytes());
  if (r) return r;
  if (!c->cp_in) {
    CK(c, cudaStreamCreateWithFlags(&c->cp_in, cudaStreamNonBlocking));
    CK(c, cudaStreamCreateWithFlags(&c->cp_out, cudaStreamNonBlocking));
  }
  std::vector<int> nch(c->cls.size());
  int total = 0;
  for (size_t k = 0; k < c->cls.size(); ++k) total += (nch[k] = std::min(c->cls[k]->ninst, c->host_chunks));
  while ((int)c->ev_in.size() < total + 1) {
    cudaEvent_t a = nullptr, b = nullptr;
    CK(c, cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    CK(c, cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    c->ev_in.push_back(a);
    c->ev_done.push_back(b);
  }
  unsigned char *dev = static_cast<unsigned char *>(c->d_stage), *hst = static_cast<unsigned char *>(psi);
  int launches = 0;
  auto queue = [&]() -> int {
    // the copies start after the work already queued on the batch's stream
    CK(c, cudaEventRecord(c->ev_done[total], c->st));
    CK(c, cudaStreamWaitEvent(c->cp_in, c->ev_done[total], 0));
    for (size_t k = 0, e = 0; k < c->cls.size(); ++k) {
      spgpe_ctx *ck = c->cls[k];
      ck->last_launches = 0;
      const size_t per = 2 * (size_t)ck->plane() * ck->es;
      for (int j = 0; j < nch[k]; ++j, ++e) {
        const int i0 = (int)((long)j * ck->ninst / nch[k]), i1 = (int)((long)(j + 1) * ck->ninst / nch[k]);
        const size_t off = c->cls_off[k] + (size_t)i0 * per, bytes = (size_t)(i1 - i0) * per;
        CK(c, cudaMemcpyAsync(dev + off, hst + off, bytes, cudaMemcpyHostToDevice, c->cp_in));
        CK(c, cudaEventRecord(c->ev_in[e], c->cp_in));
        CK(c, cudaStreamWaitEvent(ck->st, c->ev_in[e], 0));
        const int rr = run((int)k, i0, i1 - i0, dev + c->cls_off[k]);
        if (rr) return class_fail(c, ck, rr);
        CK(c, cudaEventRecord(c->ev_done[e], ck->st));
        CK(c, cudaStreamWaitEvent(c->cp_out, c->ev_done[e], 0));
        CK(c, cudaMemcpyAsync(hst + off, dev + off, bytes, cudaMemcpyDeviceToHost, c->cp_out));
      }
      launches += ck->last_launches;
    }
    return SPGPE_OK;
  };
  if ((r = queue())) {
    // copies already queued still use the caller's buffer: let them finish
    cudaStreamSynchronize(c->cp_in);
    cudaStreamSynchronize(c->cp_out);
    for (spgpe_ctx *k : c->cls) cudaStreamSynchronize(k->st);
    cudaGetLastError();
    return r;
  }
  CK(c, cudaStreamSynchronize(c->cp_out));
  for (spgpe_ctx *k : c->cls) CK(c, cudaStreamSynchronize(k->st));
  c->last_launches = launches;
  for (spgpe_ctx *k : c->cls)
    if ((r = read_flags(k))) return class_fail(c, k, r);
  return SPGPE_OK;
}

// Real-time steps of instances i0 .. i0 + ni - 1 of the batch at p, queued
// on the context's stream.
int real_enqueue(spgpe_ctx *c, void *p, double dt, int nsteps, int i0, int ni) {
  int r = ensure_tables(c, dt, 0);
  if (r) return r;
  RowArgs ra = row_args(c, p, dt);
  ColArgs ca = col_args(c, p);
  restrict_row(c, ra, i0, ni);
  restrict_col(c, ca, i0, ni);
  CK(c, row(c, kRealFirst, ra));
  for (int s = 1; s <= nsteps; ++s) {
    CK(c, col(c, false, ca));
    CK(c, row(c, s < nsteps ? kRealMid : kRealLast, ra));
  }
  return SPGPE_OK;
}

}  // namespace

extern "C" {

int spgpe_version(void) { return SPGPE_VERSION; }

const char *spgpe_last_error(const spgpe_ctx *c) { return c ? c->err.c_str() : g_init_error.c_str(); }

int spgpe_last_launches(const spgpe_ctx *c) { return c ? c->last_launches : 0; }

int spgpe_init_grid(spgpe_ctx **out, int nx, int ny, double xmax, double ymax, int dtype, void *stream) {
  return init_common(out, nx, ny, xmax, ymax, 1, dtype, stream);
}

int spgpe_init_batch(spgpe_ctx **out, int nx, int ny, double xmax, double ymax, int ninst, int dtype,
                     void *stream) {
  return init_common(out, nx, ny, xmax, ymax, ninst, dtype, stream);
}

int spgpe_init_multi(spgpe_ctx **out, int nclass, const int *nx, const int *ny, const int *ninst,
                     const double *xmax, const double *ymax, int dtype, void *stream) {
  if (!out) return fail(nullptr, SPGPE_EINVAL, "out is NULL");
  *out = nullptr;
  if (nclass < 1 || nclass > 64 || !nx || !ny || !ninst || !xmax || !ymax)
    return fail(nullptr, SPGPE_EINVAL, "nclass must be in [1, 64] and the arrays non-NULL");
  if (dtype != SPGPE_C64 && dtype != SPGPE_C128) return fail(nullptr, SPGPE_EINVAL, "dtype must be SPGPE_C64 or SPGPE_C128");
  long total = 0;
  double work = 0.0;
  for (int k = 0; k < nclass; ++k) {
    if (!pow2_in_range(nx[k]) || !pow2_in_range(ny[k]))
      return fail(nullptr, SPGPE_EINVAL, "nx and ny must be powers of two in [8, 4096]");
    if (!(std::isfinite(xmax[k]) && xmax[k] > 0 && std::isfinite(ymax[k]) && ymax[k] > 0))
      return fail(nullptr, SPGPE_EINVAL, "xmax and ymax must be finite and positive");
    if (ninst[k] < 1 || ninst[k] > 65535) return fail(nullptr, SPGPE_EINVAL, "ninst must be in [1, 65535]");
    total += ninst[k];
    work += (double)ninst[k] * nx[k] * ny[k];
  }
  if (total > 65535) return fail(nullptr, SPGPE_EINVAL, "at most 65535 instances in all");
  spgpe_ctx *c = new (std::nothrow) spgpe_ctx();
  if (!c) return fail(nullptr, SPGPE_ENOMEM, "host allocation failed");
  c->dtype = dtype;
  c->es = dtype == SPGPE_C64 ? 8 : 16;
  c->ninst = (int)total;
  c->st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 0;
  cudaGetLastError();
  auto bail = [&](int code, const std::string &msg) {
    free_all(c);
    delete c;
    return fail(nullptr, code, msg);
  };
  if (cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess)
    return bail(SPGPE_ECUDA, "cudaEventCreate failed");
  size_t off = 0;
  int first = 0;
  for (int k = 0; k < nclass; ++k) {
    cudaStream_t ks = nullptr;
    if (cudaStreamCreateWithFlags(&ks, cudaStreamNonBlocking) != cudaSuccess)
      return bail(SPGPE_ECUDA, "cudaStreamCreate failed");
    spgpe_ctx *kc = nullptr;
    const int r = init_common(&kc, nx[k], ny[k], xmax[k], ymax[k], ninst[k], dtype, ks);
    if (r) {
      cudaStreamDestroy(ks);
      return bail(r, g_init_error);
    }
    kc->own_stream = true;
    c->cls.push_back(kc);
    if (cudaEventCreateWithFlags(&kc->join_ev, cudaEventDisableTiming) != cudaSuccess)
      return bail(SPGPE_ECUDA, "cudaEventCreate failed");
    // The persistent passes of a class are sized to a share of the GPU:
    // SPGPE_CLASS_SMS=share gives each class the SMs in proportion to its
    // points, the default (full) every SM, the classes then interleaving.
    const char *mode = std::getenv("SPGPE_CLASS_SMS");
    if (sms > 0 && mode && std::strcmp(mode, "share") == 0)
      kc->sms = std::max(1, (int)std::lround(sms * (double)ninst[k] * nx[k] * ny[k] / work));
    c->cls_first.push_back(first);
    c->cls_off.push_back(off);
    first += ninst[k];
    off += kc->psi_bytes();
  }
  c->multi_bytes = off;
  c->sms = sms;
  *out = c;
  return SPGPE_OK;
}

void spgpe_destroy(spgpe_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  free_all(c);
  delete c;
}

int spgpe_set_potentials(spgpe_ctx *c, const double *V, const double *delta, const double *Omega, double g11,
                         double g22, double g12, double kL) {
  if (c && c->cls.size() > 1)
    return fail(c, SPGPE_EINVAL, "2D potential arrays need one grid size; set a multi-size batch per instance");
  if (c && c->cls.size() == 1) {
    const int r = spgpe_set_potentials(c->cls[0], V, delta, Omega, g11, g22, g12, kL);
    return r ? class_fail(c, c->cls[0], r) : r;
  }
  if (!c) return SPGPE_EINVAL;
  const size_t n = (size_t)c->nx * c->ny;
  if (!all_finite(V, n) || !all_finite(delta, n) || !all_finite(Omega, n))
    return fail(c, SPGPE_EINVAL, "potential arrays must be finite");
  const double g[4] = {g11, g22, g12, kL};
  if (!all_finite(g, 4)) return fail(c, SPGPE_EINVAL, "couplings must be finite");
  std::fill(c->hx.begin(), c->hx.end(), 0.0);
  std::fill(c->hy.begin(), c->hy.end(), 0.0);
  for (int i = 0; i < c->ninst; ++i)
    for (int k = 0; k < 4; ++k) c->hg[4 * i + k] = g[k];
  std::vector<double> p2(n * 4);
  c->vbound2d = 0.0;
  for (size_t i = 0; i < n; ++i) {
    const double v = V ? V[i] : 0.0, d = delta ? delta[i] : 0.0, o = Omega ? Omega[i] : 0.0;
    p2[4 * i] = v + 0.5 * d;
    p2[4 * i + 1] = v - 0.5 * d;
    p2[4 * i + 2] = o;
    p2[4 * i + 3] = 0.0;
    c->vbound2d = std::max(c->vbound2d, std::max(std::fabs(p2[4 * i]), std::fabs(p2[4 * i + 1])));
  }
  int r = dev_alloc(c, &c->d_pot2d, n * 2 * c->es);
  if (r) return r;
  if ((r = upload(c, c->d_pot2d, p2))) return r;
  c->has2d = true;
  c->h2d.swap(p2);
  ++c->model_version;
  if ((r = upload_raw(c))) return r;
  CK(c, cudaStreamSynchronize(c->st));
  std::fill(c->inst_set.begin(), c->inst_set.end(), 1);
  return SPGPE_OK;
}

int spgpe_set_potentials_separable(spgpe_ctx *c, int inst, const double *Vx, const double *Vy, const double *delta_x,
                                   const double *delta_y, const double *Omega_x, const double *Omega_y, double g11,
                                   double g22, double g12, double kL) {
  if (c && !c->cls.empty()) {
    if (inst == -1) {
      for (spgpe_ctx *k : c->cls)
        if (k->nx != c->cls[0]->nx || k->ny != c->cls[0]->ny)
          return fail(c, SPGPE_EINVAL, "inst = -1 needs one grid size; set a multi-size batch per instance");
      for (spgpe_ctx *k : c->cls) {
        const int r = spgpe_set_potentials_separable(k, -1, Vx, Vy, delta_x, delta_y, Omega_x, Omega_y, g11, g22,
                                                     g12, kL);
        if (r) return class_fail(c, k, r);
      }
      return SPGPE_OK;
    }
    const int k = class_of(c, inst);
    if (k < 0) return fail(c, SPGPE_EINVAL, "instance index out of range");
    const int r = spgpe_set_potentials_separable(c->cls[(size_t)k], inst - c->cls_first[(size_t)k], Vx, Vy, delta_x,
                                                 delta_y, Omega_x, Omega_y, g11, g22, g12, kL);
    return r ? class_fail(c, c->cls[(size_t)k], r) : r;
  }
  if (!c) return SPGPE_EINVAL;
  if (inst < -1 || inst >= c->ninst) return fail(c, SPGPE_EINVAL, "instance index out of range");
  const int nx = c->nx, ny = c->ny;
  if (!all_finite(Vx, nx) || !all_finite(Vy, ny) || !all_finite(delta_x, nx) || !all_finite(delta_y, ny) ||
      !all_finite(Omega_x, nx) || !all_finite(Omega_y, ny))
    return fail(c, SPGPE_EINVAL, "potential pieces must be finite");
  const double g[4] = {g11, g22, g12, kL};
  if (!all_finite(g, 4)) return fail(c, SPGPE_EINVAL, "couplings must be finite");
  ++c->model_version;
  if (c->has2d) {
    // a separable call replaces the 2D model for every instance
    c->has2d = false;
    c->vbound2d = 0.0;
    c->h2d.clear();
    if (inst >= 0) std::fill(c->inst_set.begin(), c->inst_set.end(), 0);
  }
  const int i0 = inst < 0 ? 0 : inst, i1 = inst < 0 ? c->ninst : inst + 1;
  for (int i = i0; i < i1; ++i) {
    for (int x = 0; x < nx; ++x) {
      double *h = &c->hx[((size_t)i * nx + x) * 3];
      h[0] = Vx ? Vx[x] : 0.0;
      h[1] = delta_x ? delta_x[x] : 0.0;
      h[2] = Omega_x ? Omega_x[x] : 0.0;
    }
    for (int y = 0; y < ny; ++y) {
      double *h = &c->hy[((size_t)i * ny + y) * 3];
      h[0] = Vy ? Vy[y] : 0.0;
      h[1] = delta_y ? delta_y[y] : 0.0;
      h[2] = Omega_y ? Omega_y[y] : 0.0;
    }
    for (int k = 0; k < 4; ++k) c->hg[4 * i + k] = g[k];
    c->inst_set[i] = 1;
  }
  int r = upload_raw(c);
  if (r) return r;
  CK(c, cudaStreamSynchronize(c->st));
  return SPGPE_OK;
}

int spgpe_step_real(spgpe_ctx *c, void *psi, double dt, int nsteps) {
  if (c && !c->cls.empty()) {
    if (!psi || nsteps < 0 || !std::isfinite(dt)) return fail(c, SPGPE_EINVAL, "bad psi, dt or nsteps");
    int r = check_ready(c);
    if (r) return r;
    if (nsteps > 0 && !is_device_ptr(psi))
      return host_pipeline_multi(c, psi, [&](int k, int i0, int ni, void *p) {
        return real_enqueue(c->cls[k], p, dt, nsteps, i0, ni);
      });
    return for_classes(c, psi, true, [&](spgpe_ctx *k, void *p, int) { return spgpe_step_real(k, p, dt, nsteps); });
  }
  int r = check_ready(c);
  if (r) return r;
  c->last_launches = 0;
  if (!psi || nsteps < 0 || !std::isfinite(dt)) return fail(c, SPGPE_EINVAL, "bad psi, dt or nsteps");
  if (nsteps == 0) return SPGPE_OK;
  if ((r = ensure_tables(c, dt, 0))) return r;
  // the steps of instances i0 .. i0 + ni - 1 of the batch at p
  auto run = [&](int i0, int ni, void *p) -> int { return real_enqueue(c, p, dt, nsteps, i0, ni); };
  if (!is_device_ptr(psi)) {
    if ((r = host_pipeline(c, psi, run))) return r;
    return read_flags(c);
  }
  return run(0, c->ninst, psi);
}

int spgpe_step_imag(spgpe_ctx *c, void *psi, double dtau, int nsteps, int norm_mode, const double *target,
                    double *residual_out) {
  // SPGPE_IMAG_LAGGED may be or'ed into the normalisation mode
  const bool lagged = (norm_mode & SPGPE_IMAG_LAGGED) != 0;
  norm_mode &= ~SPGPE_IMAG_LAGGED;
  if (c && !c->cls.empty()) {
    int r = check_ready(c);
    if (r) return r;
    if (!psi || nsteps < 0 || !std::isfinite(dtau)) return fail(c, SPGPE_EINVAL, "bad psi, dtau or nsteps");
    if (norm_mode != SPGPE_NORM_TOTAL && norm_mode != SPGPE_NORM_PER_COMPONENT)
      return fail(c, SPGPE_EINVAL, "bad norm_mode");
    const double t0 = target ? target[0] : 0.5, t1 = target ? target[1] : 0.5;
    if (!(std::isfinite(t0) && std::isfinite(t1) && t0 >= 0 && t1 >= 0 && t0 + t1 > 0))
      return fail(c, SPGPE_EINVAL, "targets must be finite, non-negative, not both zero");
    if (nsteps == 0) {
      if (residual_out)
        for (int i = 0; i < c->ninst; ++i) residual_out[i] = NAN;
      return SPGPE_OK;
    }
    if (!residual_out && !is_device_ptr(psi))
      return host_pipeline_multi(c, psi, [&](int k, int i0, int ni, void *p) {
        return imag_enqueue(c->cls[k], p, dtau, nsteps, norm_mode, t0, t1, false, i0, ni, lagged);
      });
    // queue every class before reading any residual, so the classes overlap
    r = for_classes(c, psi, true, [&](spgpe_ctx *k, void *p, int) {
      k->last_launches = 0;
      return imag_enqueue(k, p, dtau, nsteps, norm_mode, t0, t1, residual_out != nullptr, 0, -1, lagged);
    });
    if (r) return r;
    if (residual_out)
      for (size_t k = 0; k < c->cls.size(); ++k)
        if ((r = imag_collect(c->cls[k], dtau, residual_out + c->cls_first[k]))) return class_fail(c, c->cls[k], r);
    if (residual_out)
      for (spgpe_ctx *k : c->cls)
        if ((r = read_flags(k))) return class_fail(c, k, r);
    return SPGPE_OK;
  }
  int r = check_ready(c);
  if (r) return r;
  c->last_launches = 0;
  if (!psi || nsteps < 0 || !std::isfinite(dtau)) return fail(c, SPGPE_EINVAL, "bad psi, dtau or nsteps");
  if (norm_mode != SPGPE_NORM_TOTAL && norm_mode != SPGPE_NORM_PER_COMPONENT)
    return fail(c, SPGPE_EINVAL, "bad norm_mode");
  const double t0 = target ? target[0] : 0.5, t1 = target ? target[1] : 0.5;
  if (!(std::isfinite(t0) && std::isfinite(t1) && t0 >= 0 && t1 >= 0 && t0 + t1 > 0))
    return fail(c, SPGPE_EINVAL, "targets must be finite, non-negative, not both zero");
  if (nsteps == 0) {
    if (residual_out)
      for (int i = 0; i < c->ninst; ++i) residual_out[i] = NAN;
    return SPGPE_OK;
  }
  if (!residual_out && !is_device_ptr(psi)) {
    r = host_pipeline(c, psi, [&](int i0, int ni, void *p) {
      return imag_enqueue(c, p, dtau, nsteps, norm_mode, t0, t1, false, i0, ni, lagged);
    });
    return r ? r : read_flags(c);
  }
  void *p;
  bool host;
  if ((r = begin_psi(c, psi, &p, &host))) return r;
  if ((r = imag_enqueue(c, p, dtau, nsteps, norm_mode, t0, t1, residual_out != nullptr, 0, -1, lagged))) return r;
  if (residual_out && (r = imag_collect(c, dtau, residual_out))) return r;
  if ((r = end_psi(c, psi, host))) return r;
  if (residual_out || host) return read_flags(c);
  return SPGPE_OK;
}

int spgpe_set_timing(spgpe_ctx *c, int enable) {
  if (c)
    for (spgpe_ctx *k : c->cls) spgpe_set_timing(k, enable);
  if (!c) return SPGPE_EINVAL;
  c->timing = enable != 0;
  return SPGPE_OK;
}

int spgpe_timing(spgpe_ctx *c, double *ms_out, int *count_out) {
  if (!c || !ms_out || !count_out) return SPGPE_EINVAL;
  if (!c->cls.empty()) {
    std::vector<double> ms(SPGPE_NKINDS);
    std::vector<int> cnt(SPGPE_NKINDS);
    for (int k = 0; k < SPGPE_NKINDS; ++k) {
      ms_out[k] = 0.0;
      count_out[k] = 0;
    }
    for (spgpe_ctx *k : c->cls) {
      const int r = spgpe_timing(k, ms.data(), cnt.data());
      if (r) return class_fail(c, k, r);
      for (int j = 0; j < SPGPE_NKINDS; ++j) {
        ms_out[j] += ms[(size_t)j];
        count_out[j] += cnt[(size_t)j];
      }
    }
    return SPGPE_OK;
  }
  CK(c, cudaStreamSynchronize(c->st));
  for (int k = 0; k < SPGPE_NKINDS; ++k) {
    ms_out[k] = 0.0;
    count_out[k] = 0;
  }
  for (auto &u : c->ev_used) {
    float ms = 0.f;
    CK(c, cudaEventElapsedTime(&ms, u.second.first, u.second.second));
    ms_out[u.first] += ms;
    count_out[u.first] += 1;
    c->ev_pool.push_back(u.second.first);
    c->ev_pool.push_back(u.second.second);
  }
  c->ev_used.clear();
  return SPGPE_OK;
}

int spgpe_sync(spgpe_ctx *c) {
  if (!c) return SPGPE_EINVAL;
  if (!c->cls.empty()) {
    CK(c, cudaStreamSynchronize(c->st));
    for (spgpe_ctx *k : c->cls) {
      const int r = spgpe_sync(k);
      if (r) return class_fail(c, k, r);
    }
    return SPGPE_OK;
  }
  CK(c, cudaStreamSynchronize(c->st));
  return read_flags(c);
}

int spgpe_wait_probe(spgpe_ctx *c, long long cycles) {
  if (!c || cycles < 0) return c ? fail(c, SPGPE_EINVAL, "cycles must be >= 0") : SPGPE_EINVAL;
  spgpe_ctx *k = c->cls.empty() ? c : c->cls[0];
  CK(c, launch_wait_probe(k->d_flags, cycles, k->st));
  CK(c, cudaStreamSynchronize(k->st));
  const int r = read_flags(k);
  if (r && k != c) return class_fail(c, k, r);
  return r;
}

int spgpe_norm(spgpe_ctx *c, const void *psi, double *out) {
  if (!c || !psi || !out) return fail(c, SPGPE_EINVAL, "NULL argument");
  if (!c->cls.empty())
    return for_classes(c, psi, false, [&](spgpe_ctx *k, void *p, int first) {
      return spgpe_norm(k, p, out + 2 * (size_t)first);
    });
  void *p;
  bool host;
  int r = begin_psi(c, psi, &p, &host);
  if (r) return r;
  const int blocks = 128;
  if (c->dtype == SPGPE_C64) CK(c, launch_norm<float>(p, c->plane(), c->ninst, c->d_partials, blocks, c->st));
  else CK(c, launch_norm<double>(p, c->plane(), c->ninst, c->d_partials, blocks, c->st));
  std::vector<double> h((size_t)c->ninst * blocks * 2);
  CK(c, cudaMemcpyAsync(h.data(), c->d_partials, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  bool finite = true;
  for (int i = 0; i < c->ninst; ++i) {
    double su = 0, sd = 0;
    for (int b = 0; b < blocks; ++b) {
      su += h[((size_t)i * blocks + b) * 2];
      sd += h[((size_t)i * blocks + b) * 2 + 1];
    }
    out[2 * i] = su * c->dx * c->dy;
    out[2 * i + 1] = sd * c->dx * c->dy;
    finite = finite && std::isfinite(out[2 * i]) && std::isfinite(out[2 * i + 1]);
  }
  return finite ? SPGPE_OK : fail(c, SPGPE_ENONFINITE, "non-finite atom number");
}

int spgpe_energy(spgpe_ctx *c, const void *psi, double *out) {
  int r = check_ready(c);
  if (r) return r;
  if (!psi || !out) return fail(c, SPGPE_EINVAL, "NULL argument");
  if (!c->cls.empty())
    return for_classes(c, psi, false, [&](spgpe_ctx *k, void *p, int first) {
      return spgpe_energy(k, p, out + 6 * (size_t)first);
    });
  if ((r = dev_alloc(c, &c->d_scratch, c->psi_bytes()))) return r;
  void *p;
  bool host;
  if ((r = begin_psi(c, psi, &p, &host))) return r;
  EnergyArgs a{};
  a.psi = p;
  a.scratch = c->d_scratch;
  a.rawx = c->d_rawx;
  a.rawy = c->d_rawy;
  a.pot2d = c->has2d ? c->d_pot2d : nullptr;
  a.twx = c->d_twe ? c->d_twe : c->d_twx;
  a.twy = c->d_twy;
  a.gpar = c->d_gpar;
  a.partials = c->d_partials;
  a.dkx = kTwoPi / (c->nx * c->dx);
  a.dky = kTwoPi / (c->ny * c->dy);
  a.nx = c->nx;
  a.ny = c->ny;
  a.ninst = c->ninst;
  int rb = 0, cb = 0;
  if (c->dtype == SPGPE_C64) CK(c, launch_energy<float>(a, c->st, &rb, &cb));
  else CK(c, launch_energy<double>(a, c->st, &rb, &cb));
  const size_t nrow = (size_t)c->ninst * rb * 6, ncol = (size_t)c->ninst * 2 * cb;
  std::vector<double> h(nrow + ncol);
  CK(c, cudaMemcpyAsync(h.data(), c->d_partials, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  const double w = c->dx * c->dy;
  bool finite = true;
  for (int i = 0; i < c->ninst; ++i) {
    double s[6] = {0, 0, 0, 0, 0, 0}, kin = 0;
    for (int b = 0; b < rb; ++b)
      for (int k = 0; k < 6; ++k) s[k] += h[((size_t)i * rb + b) * 6 + k];
    for (int j = 0; j < 2; ++j)
      for (int b = 0; b < cb; ++b) kin += h[nrow + ((size_t)i * 2 + j) * cb + b];
    double *o = out + 6 * (size_t)i;
    o[1] = kin * w / ((double)c->nx * c->ny);
    o[2] = s[0] * w;
    o[3] = s[1] * w;
    o[4] = s[2] * w;
    o[5] = s[3] * w;
    o[0] = o[1] + o[2] + o[3] + o[4] + o[5];
    for (int k = 0; k < 6; ++k) finite = finite && std::isfinite(o[k]);
  }
  return finite ? SPGPE_OK : fail(c, SPGPE_ENONFINITE, "non-finite energy");
}

int spgpe_cufft_step_real(spgpe_ctx *c, void *psi, double dt, int nsteps) {
  if (c && !c->cls.empty()) {
    if (!psi || !is_device_ptr(psi)) return fail(c, SPGPE_EINVAL, "the comparator takes device spinors only");
    return for_classes(c, psi, false, [&](spgpe_ctx *k, void *p, int) {
      return spgpe_cufft_step_real(k, p, dt, nsteps);
    });
  }
  int r = check_ready(c);
  if (r) return r;
  c->last_launches = 0;
  if (!psi || nsteps < 0 || !std::isfinite(dt)) return fail(c, SPGPE_EINVAL, "bad psi, dt or nsteps");
  if (!is_device_ptr(psi)) return fail(c, SPGPE_EINVAL, "the comparator takes device spinors only");
  if (nsteps == 0) return SPGPE_OK;
  if ((r = ensure_tables(c, dt, 0))) return r;
  if (!c->plan_ok) {
    int n[2] = {c->ny, c->nx};
    const cufftType ty = c->dtype == SPGPE_C64 ? CUFFT_C2C : CUFFT_Z2Z;
    if (cufftPlanMany(&c->plan, 2, n, nullptr, 1, 0, nullptr, 1, 0, ty, 2 * c->ninst) != CUFFT_SUCCESS)
      return fail(c, SPGPE_ECUDA, "cufftPlanMany failed");
    c->plan_ok = true;
  }
  if (cufftSetStream(c->plan, c->st) != CUFFT_SUCCESS) return fail(c, SPGPE_ECUDA, "cufftSetStream failed");
  const RowArgs ra = row_args(c, psi, dt);
  const ColArgs ca = col_args(c, psi);
  for (int s = 0; s < nsteps; ++s) {
    if (c->dtype == SPGPE_C64) {
      CK(c, launch_ref_R<float>(false, ra, c->st));
      if (cufftExecC2C(c->plan, (cufftComplex *)psi, (cufftComplex *)psi, CUFFT_FORWARD) != CUFFT_SUCCESS)
        return fail(c, SPGPE_ECUDA, "cufftExecC2C failed");
      CK(c, launch_ref_K<float>(ca, c->st));
      if (cufftExecC2C(c->plan, (cufftComplex *)psi, (cufftComplex *)psi, CUFFT_INVERSE) != CUFFT_SUCCESS)
        return fail(c, SPGPE_ECUDA, "cufftExecC2C failed");
      CK(c, launch_ref_R<float>(false, ra, c->st));
    } else {
      CK(c, launch_ref_R<double>(false, ra, c->st));
      if (cufftExecZ2Z(c->plan, (cufftDoubleComplex *)psi, (cufftDoubleComplex *)psi, CUFFT_FORWARD) != CUFFT_SUCCESS)
        return fail(c, SPGPE_ECUDA, "cufftExecZ2Z failed");
      CK(c, launch_ref_K<double>(ca, c->st));
      if (cufftExecZ2Z(c->plan, (cufftDoubleComplex *)psi, (cufftDoubleComplex *)psi, CUFFT_INVERSE) != CUFFT_SUCCESS)
        return fail(c, SPGPE_ECUDA, "cufftExecZ2Z failed");
      CK(c, launch_ref_R<double>(false, ra, c->st));
    }
    c->last_launches += 3;
  }
  return SPGPE_OK;
}

}  // extern "C"

// ------------------------------------------------ relaxation to a tolerance

namespace {

// The complex64 twin of a complex128 context (same grid, batch, stream and
// model) and its spinor buffer, brought up to date with the model.
int ensure_twin(spgpe_ctx *c) {
  if (!c->twin) {
    spgpe_ctx *t = nullptr;
    const int r = init_common(&t, c->nx, c->ny, c->xmax, c->ymax, c->ninst, SPGPE_C64, c->st);
    if (r) return fail(c, r, "complex64 twin: " + g_init_error);
    t->persistent_row = c->persistent_row;
    t->persistent_col = c->persistent_col;
    t->warp_col = c->warp_col;
    c->twin = t;
  }
  spgpe_ctx *t = c->twin;
  if (c->twin_version != c->model_version) {
    t->hx = c->hx;
    t->hy = c->hy;
    t->hg = c->hg;
    t->inst_set = c->inst_set;
    t->has2d = c->has2d;
    t->vbound2d = c->vbound2d;
    t->h2d = c->h2d;
    int r = SPGPE_OK;
    if (t->has2d) {
      if ((r = dev_alloc(t, &t->d_pot2d, (size_t)c->nx * c->ny * 2 * t->es)) || (r = upload(t, t->d_pot2d, t->h2d)))
        return fail(c, r, "complex64 twin: " + t->err);
    }
    if ((r = upload_raw(t))) return fail(c, r, "complex64 twin: " + t->err);
    c->twin_version = c->model_version;
  }
  return dev_alloc(c, &c->d_psi64, t->psi_bytes());
}

// A context that owns kernels (a single-size context, a size class of a
// multi-size batch, or their complex64 twins), its device spinor and the
// global index of its first instance.
struct Member {
  spgpe_ctx *c;
  void *p;
  int first;
};

// Imaginary-time steps in chunks of `check`, each ending with the residual of
// its last step, until every instance is within tol or max_steps have run.
// The members' chunks are queued on their own streams before any residual is
// read, so size classes run side by side.  An instance that is done is frozen
// (the passes skip it) while the others go on; its residual stays the last
// one measured.  to_floor: an instance also stops holding the stage open once
// its residual has reached the rounding floor of complex64 (below 2^-18 /
// dtau) and improves by less than a fifth from one chunk to the next, but is
// stepped on until the stage ends (its slow modes keep relaxing; the stage
// budget is shared with the next one).  give_up: an instance is also
// done once its smallest residual so far has not halved in kStallChecks
// chunks (a metastable state, or a relaxation far too slow for the budget).
constexpr int kStallChecks = 40;
int relax_stage(spgpe_ctx *owner, std::vector<Member> &mem, int ntotal, double dtau, double tol, int max_steps,
                int check, int norm_mode, double t0, double t1, bool to_floor, bool give_up, bool lagged,
                std::vector<double> &res, int *steps, int *launches) {
  const double floor64 = std::ldexp(1.0, -18) / dtau;
  std::vector<int> act((size_t)ntotal, 1), since((size_t)ntotal, 0);
  std::vector<char> counted((size_t)ntotal, 0);  // no longer holding the stage open
  std::vector<double> prev((size_t)ntotal, INFINITY), best((size_t)ntotal, INFINITY), r((size_t)ntotal);
  int done = 0, nact = ntotal;
  auto upload_mask = [&](const Member &m) {
    return cudaMemcpyAsync(m.c->d_active, act.data() + m.first, (size_t)m.c->ninst * sizeof(int),
                           cudaMemcpyHostToDevice, m.c->st);
  };
  auto finish = [&](int code) {
    for (Member &m : mem) m.c->use_active = false;
    *steps = done;
    return code;
  };
  for (Member &m : mem) {
    const cudaError_t e = upload_mask(m);
    if (e != cudaSuccess) return finish(cuda_fail(owner, e, "active mask upload"));
    m.c->use_active = true;
  }
  // Chunks after the first are replayed from a CUDA graph of the whole chunk
  // (every member, forked from and joined into the owner's stream); the
  // frozen-instance mask is read from device memory, so the graph stays valid.
  const bool multi = !owner->cls.empty();
  const cudaStream_t os = multi ? owner->st : mem[0].c->st;
  bool timing = false;
  for (Member &m : mem) timing = timing || m.c->timing;
  cudaGraphExec_t exec = nullptr;
  int graph_launches = 0;
  // the legacy and per-thread default streams cannot be captured
  bool use_graph = os != nullptr && os != cudaStreamLegacy && os != cudaStreamPerThread;
  auto enqueue = [&](int n) -> int {
    int rc;
    if (multi && (rc = fork_classes(owner))) return rc;
    for (Member &m : mem) {
      m.c->last_launches = 0;
      if ((rc = imag_enqueue(m.c, m.p, dtau, n, norm_mode, t0, t1, true, 0, -1, lagged)))
        return fail(owner, rc, m.c->err);
      graph_launches += m.c->last_launches;
    }
    if (multi && (rc = join_classes(owner))) return rc;
    return SPGPE_OK;
  };
  auto drop_graph = [&] {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
  };
  while (done < max_steps && nact > 0) {
    const int n = std::min(check, max_steps - done);
    int rc = SPGPE_OK;
    if (done > 0 && n == check && !timing && use_graph && !exec) {
      // capture one chunk (tables, scratch and launch attributes are in place
      // after the first); if capture is refused, run the chunks directly
      cudaGraph_t g = nullptr;
      graph_launches = 0;
      bool ok = cudaStreamBeginCapture(os, cudaStreamCaptureModeRelaxed) == cudaSuccess;
      if (ok) {
        const int rc0 = enqueue(n);
        ok = cudaStreamEndCapture(os, &g) == cudaSuccess && rc0 == SPGPE_OK && g &&
             cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
      }
      if (!ok) {
        drop_graph();
        use_graph = false;
        cudaGetLastError();
        owner->err.clear();
      }
    }
    if (exec && n == check) {
      const cudaError_t e = cudaGraphLaunch(exec, os);
      if (e != cudaSuccess) {
        drop_graph();
        return finish(cuda_fail(owner, e, "cudaGraphLaunch"));
      }
      *launches += graph_launches;
      if (multi) {
        const cudaError_t e3 = cudaStreamSynchronize(os);  // the members' streams read what the graph wrote
        if (e3 != cudaSuccess) {
          drop_graph();
          return finish(cuda_fail(owner, e3, "chunk graph"));
        }
      }
    } else {
      graph_launches = 0;
      rc = enqueue(n);
      *launches += graph_launches;
      if (rc) {
        drop_graph();
        return finish(rc);
      }
    }
    for (Member &m : mem) {
      rc = imag_collect(m.c, dtau, r.data() + m.first);
      if (!rc) rc = read_flags(m.c);
      if (rc) {
        drop_graph();
        return finish(fail(owner, rc, m.c->err));
      }
    }
    done += n;
    std::vector<char> changed(mem.size(), 0);
    for (size_t k = 0; k < mem.size(); ++k)
      for (int j = 0; j < mem[k].c->ninst; ++j) {
        const size_t i = (size_t)(mem[k].first + j);
        if (!act[i]) continue;
        const double v = std::isnan(r[i]) ? INFINITY : r[i];
        res[i] = v;
        if (v < 0.5 * best[i]) {
          best[i] = v;
          since[i] = 0;
        } else {
          ++since[i];
        }
        if (v <= tol || (give_up && since[i] >= kStallChecks)) {
          act[i] = 0;
          changed[k] = 1;
          if (!counted[i]) {
            counted[i] = 1;
            --nact;
          }
        } else if (to_floor && !counted[i] && v < floor64 && v > 0.8 * prev[i]) {
          // at the floor: done for this stage, but stepped on while the stage
          // lasts (cheap in complex64), so that its slow modes keep relaxing
          counted[i] = 1;
          --nact;
        }
        prev[i] = v;
      }
    if (nact > 0)
      for (size_t k = 0; k < mem.size(); ++k)
        if (changed[k]) {
          // a pageable-memory copy: the host array is consumed before the call
          // returns; a multi-size batch's graph runs on another stream, so the
          // copy must also have landed
          cudaError_t e = upload_mask(mem[k]);
          if (e == cudaSuccess && multi) e = cudaStreamSynchronize(mem[k].c->st);
          if (e != cudaSuccess) {
            drop_graph();
            return finish(cuda_fail(owner, e, "active mask upload"));
          }
        }
  }
  drop_graph();
  return finish(SPGPE_OK);
}

}  // namespace

extern "C" int spgpe_relax(spgpe_ctx *c, void *psi, double dtau, double tol, int max_steps, int check_every,
                           int norm_mode, const double *target, int flags, double handoff, double *residual_out,
                           int *steps_out) {
  int r = check_ready(c);
  if (r) return r;
  c->last_launches = 0;
  if (!psi || !(dtau > 0) || !std::isfinite(dtau) || !(tol > 0) || max_steps < 1 || check_every < 1 ||
      !(handoff >= 0) || !std::isfinite(handoff))
    return fail(c, SPGPE_EINVAL, "bad psi, dtau, tol, max_steps, check_every or handoff");
  if (flags & ~(SPGPE_RELAX_LADDER | SPGPE_RELAX_GIVE_UP | SPGPE_RELAX_LAGGED))
    return fail(c, SPGPE_EINVAL, "unknown flags");
  if (norm_mode != SPGPE_NORM_TOTAL && norm_mode != SPGPE_NORM_PER_COMPONENT)
    return fail(c, SPGPE_EINVAL, "bad norm_mode");
  const double t0 = target ? target[0] : 0.5, t1 = target ? target[1] : 0.5;
  if (!(std::isfinite(t0) && std::isfinite(t1) && t0 >= 0 && t1 >= 0 && t0 + t1 > 0))
    return fail(c, SPGPE_EINVAL, "targets must be finite, non-negative, not both zero");
  const bool ladder = (flags & SPGPE_RELAX_LADDER) && c->dtype == SPGPE_C128;
  const bool give_up = (flags & SPGPE_RELAX_GIVE_UP) != 0;
  const bool lagged = (flags & SPGPE_RELAX_LAGGED) != 0;
  void *p;
  bool host;
  if ((r = begin_psi(c, psi, &p, &host))) return r;
  std::vector<Member> mem;
  if (c->cls.empty()) {
    mem.push_back({c, p, 0});
  } else {
    if ((r = fork_classes(c))) return r;
    for (size_t k = 0; k < c->cls.size(); ++k)
      mem.push_back({c->cls[k], static_cast<char *>(p) + c->cls_off[k], c->cls_first[k]});
  }
  std::vector<double> res((size_t)c->ninst, NAN);
  int s64 = 0, s = 0, launches = 0;
  if (ladder) {
    std::vector<Member> m64;
    for (Member &m : mem) {
      if ((r = ensure_twin(m.c))) return fail(c, r, m.c->err);
      CK(c, launch_convert(m.p, 16, m.c->d_psi64, 8, (long)m.c->ninst * 2 * m.c->plane(), m.c->sms, m.c->st));
      m64.push_back({m.c->twin, m.c->d_psi64, m.first});
      ++launches;
    }
    // complex64 down to the hand-off residual, or (handoff = 0) its rounding floor
    r = relax_stage(c, m64, c->ninst, dtau, std::max(tol, handoff), max_steps, check_every, norm_mode, t0, t1,
                    handoff == 0.0, give_up, lagged, res, &s64, &launches);
    if (r) return r;
    for (Member &m : mem) {
      CK(c, launch_convert(m.c->d_psi64, 8, m.p, 16, (long)m.c->ninst * 2 * m.c->plane(), m.c->sms, m.c->st));
      ++launches;
    }
  }
  // the context's own precision (a staged host spinor is already on the device),
  // with what is left of the step budget
  const int left = std::max(0, max_steps - s64);
  if (left > 0)
    r = relax_stage(c, mem, c->ninst, dtau, tol, left, check_every, norm_mode, t0, t1, false, give_up, lagged,
                    res, &s, &launches);
  if (r) return r;
  if (!c->cls.empty() && (r = join_classes(c))) return r;
  c->last_launches = launches;
  if ((r = end_psi(c, psi, host))) return r;
  if (residual_out)
    for (int i = 0; i < c->ninst; ++i) residual_out[i] = res[(size_t)i];
  if (steps_out) {
    steps_out[0] = s64;
    steps_out[1] = s;
  }
  return SPGPE_OK;
}

// ------------------------------------------------------------- autotuning

extern "C" int spgpe_autotune(spgpe_ctx *c, const void *psi, double dt, int *choice_out, double *ms_out) {
  int r = check_ready(c);
  if (r) return r;
  if (!psi || !std::isfinite(dt)) return fail(c, SPGPE_EINVAL, "bad psi or dt");
  void *p;
  bool host;
  if ((r = begin_psi(c, psi, &p, &host))) return r;
  std::vector<Member> mem;
  if (c->cls.empty()) {
    mem.push_back({c, p, 0});
  } else {
    CK(c, cudaStreamSynchronize(c->st));  // the spinor's producers are done before the classes copy it
    for (size_t k = 0; k < c->cls.size(); ++k)
      mem.push_back({c->cls[k], static_cast<char *>(p) + c->cls_off[k], c->cls_first[k]});
  }
  constexpr int kWarm = 3, kTimed = 16, kReps = 2;
  for (size_t k = 0; k < mem.size(); ++k) {
    spgpe_ctx *m = mem[k].c;
    if ((r = dev_alloc(m, &m->d_scratch, m->psi_bytes()))) return fail(c, r, m->err);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    // each variant timed kReps times, the variants interleaved; the minimum
    // counts.  Variant v: bit 0 persistent row pass; v >> 1 the column pass
    // (0 plain, 1 persistent TMA, 2 warp-local, where it applies).
    const int nv = warp_col_applies(m) ? 6 : 4;
    float vms[6] = {INFINITY, INFINITY, INFINITY, INFINITY, INFINITY, INFINITY};
    auto set_variant = [](spgpe_ctx *x, int v) {
      x->persistent_row = (v & 1) != 0;
      x->persistent_col = (v >> 1) == 1;
      x->warp_col = (v >> 1) == 2;
    };
    for (int rep = 0; rep < kReps && !r; ++rep)
      for (int v = 0; v < nv && !r; ++v) {
        set_variant(m, v);
        cudaError_t e = cudaMemcpyAsync(m->d_scratch, mem[k].p, m->psi_bytes(), cudaMemcpyDeviceToDevice, m->st);
        if (e != cudaSuccess) {
          r = cuda_fail(c, e, "autotune copy");
          break;
        }
        if ((r = spgpe_step_real(m, m->d_scratch, dt, kWarm))) break;
        float ms = 0.f;
        if ((e = cudaEventRecord(e0, m->st)) != cudaSuccess) {
          r = cuda_fail(c, e, "autotune timing");
          break;
        }
        if ((r = spgpe_step_real(m, m->d_scratch, dt, kTimed))) break;
        if ((e = cudaEventRecord(e1, m->st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
          r = cuda_fail(c, e, "autotune timing");
          break;
        }
        vms[v] = std::min(vms[v], ms);
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) return r == SPGPE_ECUDA ? r : fail(c, r, m->err);
    int best = 0;
    for (int v = 1; v < nv; ++v)
      if (vms[v] < vms[best]) best = v;
    const float best_ms = vms[best];
    set_variant(m, best);
    if (m->twin) set_variant(m->twin, best);
    if (choice_out) choice_out[k] = best;
    if (ms_out) ms_out[k] = best_ms / kTimed;
  }
  if (host) CK(c, cudaStreamSynchronize(c->st));
  return SPGPE_OK;
}

// ------------------------------------------- Sec. 6 observables and noise

namespace {

int observables_one(spgpe_ctx *c, void *p, double *out) {
  ObsGeom g;
  g.nx = c->nx;
  g.ny = c->ny;
  g.xmax = c->xmax;
  g.ymax = c->ymax;
  g.dx = c->dx;
  g.dy = c->dy;
  g.h = 0.5 * std::min(c->dx, c->dy);
  g.nb = (int)(std::sqrt(c->xmax * c->xmax + c->ymax * c->ymax) / g.h) + 2;
  const int ni = c->ninst, sb = 128, npts = 4 * std::max(c->nx, c->ny);
  // [ninst][nb] histogram, then R [ninst] and windings [ninst][2]
  const size_t need = (size_t)ni * ((size_t)g.nb + 3);
  if (c->n_obs < need) {
    if (c->d_obs) cudaFree(c->d_obs);
    c->d_obs = nullptr;
    c->n_obs = 0;
    const int r = dev_alloc(c, (void **)&c->d_obs, need * sizeof(double));
    if (r) return r;
    c->n_obs = need;
  }
  double *hist = c->d_obs, *dR = hist + (size_t)ni * g.nb, *dw = dR + ni;
  CK(c, cudaMemsetAsync(hist, 0, (size_t)ni * g.nb * sizeof(double), c->st));
  CK(c, launch_observables((int)c->es, p, g, ni, c->d_partials, sb, hist, nullptr, npts, nullptr, 0, c->st));
  std::vector<double> part((size_t)ni * sb * 4), h((size_t)ni * g.nb);
  CK(c, cudaMemcpyAsync(part.data(), c->d_partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaMemcpyAsync(h.data(), hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  std::vector<double> R((size_t)ni);
  for (int i = 0; i < ni; ++i) {
    double a = 0, b = 0, cc = 0, tot = 0;
    for (int k = 0; k < sb; ++k) {
      const double *q = &part[((size_t)i * sb + k) * 4];
      a += q[0];
      b += q[1];
      cc += q[2];
      tot += q[3];
    }
    out[4 * (size_t)i] = 1.0 - a / std::sqrt(b * cc);
    // the radius whose bins first hold 99 % of the atoms
    double cum = 0.0, rr = g.nb * g.h;
    for (int k = 0; k < g.nb; ++k) {
      cum += h[(size_t)i * g.nb + k];
      if (cum >= 0.99 * tot) {
        rr = (k + 1) * g.h;
        break;
      }
    }
    R[(size_t)i] = rr;
    out[4 * (size_t)i + 3] = rr;
  }
  CK(c, cudaMemcpyAsync(dR, R.data(), R.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(c, launch_observables((int)c->es, p, g, ni, nullptr, sb, nullptr, dR, npts, dw, 1, c->st));
  std::vector<double> w((size_t)ni * 2);
  CK(c, cudaMemcpyAsync(w.data(), dw, w.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(c, cudaStreamSynchronize(c->st));
  bool finite = true;
  for (int i = 0; i < ni; ++i) {
    out[4 * (size_t)i + 1] = w[2 * (size_t)i];
    out[4 * (size_t)i + 2] = w[2 * (size_t)i + 1];
    for (int k = 0; k < 4; ++k) finite = finite && std::isfinite(out[4 * (size_t)i + k]);
  }
  return finite ? SPGPE_OK : fail(c, SPGPE_ENONFINITE, "non-finite observable");
}

}  // namespace

extern "C" int spgpe_observables(spgpe_ctx *c, const void *psi, double *out) {
  if (!c || !psi || !out) return fail(c, SPGPE_EINVAL, "NULL argument");
  if (!c->cls.empty())
    return for_classes(c, psi, false, [&](spgpe_ctx *k, void *p, int first) {
      return spgpe_observables(k, p, out + 4 * (size_t)first);
    });
  void *p;
  bool host;
  int r = begin_psi(c, psi, &p, &host);
  if (r) return r;
  return observables_one(c, p, out);
}

extern "C" int spgpe_add_noise(spgpe_ctx *c, void *psi, double sigma, unsigned long long seed) {
  if (!c || !psi) return fail(c, SPGPE_EINVAL, "NULL argument");
  if (!(sigma >= 0) || !std::isfinite(sigma)) return fail(c, SPGPE_EINVAL, "sigma must be finite and >= 0");
  auto one = [&](spgpe_ctx *k, void *p, int first) -> int {
    const cudaError_t e = launch_add_noise((int)k->es, p, 2L * k->nx * k->ny, k->ninst, first, sigma, seed,
                                           std::max(1, k->sms), k->st);
    k->last_launches = 1;
    return e == cudaSuccess ? SPGPE_OK : cuda_fail(k, e, "add_noise");
  };
  if (!c->cls.empty()) return for_classes(c, psi, true, one);
  void *p;
  bool host;
  int r = begin_psi(c, psi, &p, &host);
  if (r) return r;
  if ((r = one(c, p, 0))) return r;
  return end_psi(c, psi, host);
}
