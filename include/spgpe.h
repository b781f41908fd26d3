/*
 * spgpe.h -- C ABI of the GB300 (sm_103a) time-splitting spectral solver for
 * the two-component quasi-2D Gross-Pitaevskii equation of arXiv:2010.15069.
 *
 * Model (Eq. 3 signs, hbar = m = omega_perp = 1; Eqs. 4-8 split it into the
 * kinetic H(1), potential H(2), interaction H(3) and Raman H(4) parts):
 *
 *   i dPsi/dt = H Psi,  Psi = (psi_up, psi_dn),
 *   H = diag(T_up, T_dn)(k) + V 1 + (delta/2) sigma_z + (Omega/2) sigma_x
 *       + diag(g11 rho_up + g12 rho_dn, g22 rho_dn + g12 rho_up),
 *   T_up(k) = k^2/2 - kL kx,   T_dn(k) = k^2/2 + kL kx,   rho_j = |psi_j|^2.
 *
 * Grid (Sec. 3.2): x_i = -xmax + i dx, dx = 2 xmax / nx (periodic, +xmax
 * excluded), kx = 2 pi fftfreq(nx, dx) with the Nyquist bin at -pi/dx; the
 * same in y.  nx and ny are powers of two in [8, 4096].
 *
 * One step (Eq. 13 operators, Strang splitting of Sec. 3.2, four 2D FFTs):
 *   S(dt) = R(dt/2) F^-1 K(dt) F R(dt/2),   R(tau) = X(tau/2) D(tau) X(tau/2),
 *   D(tau): psi_up *= exp(-i tau (V + delta/2 + g11 rho_up + g12 rho_dn)),
 *           psi_dn *= exp(-i tau (V - delta/2 + g22 rho_dn + g12 rho_up)),
 *           densities taken on entry to D;
 *   X(tau) = exp(-i tau Omega sigma_x / 2);  K(tau): psi_hat_j *= exp(-i tau T_j(k)).
 * Imaginary time replaces -i tau by -tau in every factor and rescales the
 * spinor to the target atom number after every step (Sec. 3.2).
 *
 * Data layout: a spinor batch is [ninst][2][ny][nx] interleaved complex
 * (re, im), component up first, x fastest, in the context's precision
 * (SPGPE_C64: float pairs, SPGPE_C128: double pairs).  Atom numbers are
 * N_j = dx dy sum |psi_j|^2.
 *
 * Ownership and threading: the spinor buffer and the CUDA stream belong to
 * the caller; tables, twiddles and scratch belong to the context.  A context
 * is not thread-safe; use one context per stream.  Calls on device buffers
 * are stream-ordered and asynchronous unless documented as synchronising.
 *
 * Errors: every call returns SPGPE_OK (0) or a negative status; nothing is
 * thrown or aborted across the ABI.  spgpe_last_error() gives a message.
 */
#ifndef SPGPE_H
#define SPGPE_H

#ifdef __cplusplus
extern "C" {
#endif

#define SPGPE_VERSION 100

enum { SPGPE_C64 = 1, SPGPE_C128 = 2 };
enum { SPGPE_NORM_TOTAL = 0, SPGPE_NORM_PER_COMPONENT = 1 };
/* Or'ed into the norm_mode of spgpe_step_imag: the lagged renormalisation
 * (see there). */
enum { SPGPE_IMAG_LAGGED = 4 };
enum {
  SPGPE_OK = 0,
  SPGPE_EINVAL = -1,     /* bad argument: size, pointer, dtype, non-finite input */
  SPGPE_ENOMEM = -2,     /* device or host allocation failed */
  SPGPE_ECUDA = -3,      /* a CUDA runtime call failed; see spgpe_last_error */
  SPGPE_ENONFINITE = -4, /* a norm or energy reduction met NaN/Inf (or a zero norm) */
  SPGPE_ETIMEOUT = -5,   /* a bounded device wait gave up (a tile transfer never landed) */
  SPGPE_ESTATE = -6,     /* call out of order (e.g. stepping before potentials) */
  SPGPE_EBOUNDS = -7     /* an index fell outside its buffer (bounds-checked builds only) */
};

typedef struct spgpe_ctx spgpe_ctx;

/* Create a context for one nx x ny instance over [-xmax, xmax) x [-ymax, ymax)
 * (Sec. 3.2 grid).  dtype is SPGPE_C64 or SPGPE_C128.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream), borrowed, not owned.  Allocates
 * the context's device tables.  Returns EINVAL for sizes that are not powers
 * of two in [8, 4096], non-positive or non-finite extents, or a bad dtype;
 * ENOMEM / ECUDA on allocation failure.  *out is NULL on failure. */
int spgpe_init_grid(spgpe_ctx **out, int nx, int ny, double xmax, double ymax,
                    int dtype, void *cuda_stream);

/* As spgpe_init_grid for a batch of ninst (>= 1) independent instances of the
 * same grid, each with its own potentials and couplings (parameter sweeps).
 * The spinor buffer then holds ninst spinors back to back. */
int spgpe_init_batch(spgpe_ctx **out, int nx, int ny, double xmax, double ymax,
                     int ninst, int dtype, void *cuda_stream);

/* A batch over several grid sizes (parameter sweeps over grids, e.g. 64
 * instances at 256^2 with 16 at 512^2 and 4 at 1024^2).  Size class k holds
 * ninst[k] instances of an nx[k] x ny[k] grid over [-xmax[k], xmax[k]) x
 * [-ymax[k], ymax[k]); instances are numbered class by class, and the spinor
 * buffer holds them back to back in that order, each [2][ny][nx].  Each
 * class runs on a CUDA stream of its own, started after the work already on
 * cuda_stream and joined back into it, so the classes of one call run side
 * by side, their persistent passes sharing the SMs in proportion to their
 * points.  Every call below accepts such a context: instance indices and
 * per-instance outputs are global; spgpe_set_potentials (2D arrays) and
 * spgpe_set_potentials_separable with inst = -1 need all classes of one
 * size.  nclass in [1, 64], at most 65535 instances in all. */
int spgpe_init_multi(spgpe_ctx **out, int nclass, const int *nx, const int *ny, const int *ninst,
                     const double *xmax, const double *ymax, int dtype, void *cuda_stream);

/* Potentials and couplings of Eqs. 3-8 for every instance.  V, delta, Omega
 * are host FP64 arrays [ny][nx] (row-major), NULL meaning zero; they are
 * copied (the caller may free them on return) and stored in the working
 * precision.  g11, g22, g12 are the interaction strengths, kL the Raman
 * recoil momentum of the kL kx sigma_z term.  Synchronises the stream.
 * Returns EINVAL on a NULL context or any non-finite value. */
int spgpe_set_potentials(spgpe_ctx *ctx, const double *V, const double *delta,
                         const double *Omega, double g11, double g22, double g12,
                         double kL);

/* Separable form of the same call that moves no 2D arrays:
 * V(x,y) = Vx[ix] + Vy[iy], delta = delta_x[ix] + delta_y[iy],
 * Omega = Omega_x[ix] + Omega_y[iy]; each pointer is a host FP64 array of
 * length nx (x pieces) or ny (y pieces), NULL meaning zero.  inst selects the
 * instance of a batch; inst = -1 sets every instance.  Replaces any 2D arrays
 * given earlier.  Synchronises the stream.  EINVAL on bad inst or non-finite
 * values. */
int spgpe_set_potentials_separable(spgpe_ctx *ctx, int inst, const double *Vx,
                                   const double *Vy, const double *delta_x,
                                   const double *delta_y, const double *Omega_x,
                                   const double *Omega_y, double g11, double g22,
                                   double g12, double kL);

/* nsteps real-time Strang steps S(dt) in place on psi (Sec. 3.2, Fig. 1
 * loop).  psi is the caller's [ninst][2][ny][nx] complex buffer in the
 * context's precision.  A device pointer is updated asynchronously on the
 * stream; a host pointer is copied in, stepped and copied back before the
 * call returns (synchronising).  The state on return equals nsteps
 * applications of S(dt); consecutive R(dt/2) halves are fused only inside
 * the call, so a run split over several calls gives the same bits.
 * nsteps = 0 is a no-op.  ESTATE before any set_potentials call. */
int spgpe_step_real(spgpe_ctx *ctx, void *psi, double dt, int nsteps);

/* nsteps imaginary-time steps (dt -> -i dtau), rescaling after every step to
 * the target atom numbers (Sec. 3.2): norm_mode SPGPE_NORM_TOTAL scales both
 * components by sqrt((target[0]+target[1]) / (N_up+N_dn)),
 * SPGPE_NORM_PER_COMPONENT scales psi_j by sqrt(target[j] / N_j).  target is a
 * host array of 2 doubles shared by all instances (NULL = {0.5, 0.5}).
 *
 * Placement of the rescaling.  By default every step is S(dtau) followed by
 * the exact rescaling (the definition above; three passes over psi per step).
 * With SPGPE_IMAG_LAGGED or'ed into norm_mode, the step boundaries after the
 * first (except the one into the last step when residual_out is given) take
 * two passes: the opening R(dtau/2) of step n+1 runs on the closing result of
 * step n scaled by the previous boundary's scale s_{n-1}, and the column pass
 * that follows multiplies by s_n / s_{n-1}, s_n being the exact scale of step
 * n.  The linear part of the rescaling is then exact and only the densities
 * in the opening D(dtau/2) lag: a stationary state of one map is a
 * stationary state of the other (s_n = s_{n-1} there), so both relax to the
 * same ground state, while the states of a transient differ at O(dtau g rho
 * (s_n^2 / s_{n-1}^2 - 1)).  The first boundary and the end of the call are
 * exact, so the state on return is normalised.
 * residual_out (host, nullable; ninst doubles) receives the discrete-map
 * residual of the last step, ||Psi_{n+1} - Psi_n||_2 / (dtau ||Psi_n||_2)
 * over both components; asking for it synchronises.  A NaN/Inf or zero norm
 * met during the run is reported as ENONFINITE by the next synchronising
 * call (this one when residual_out is given). */
int spgpe_step_imag(spgpe_ctx *ctx, void *psi, double dtau, int nsteps, int norm_mode,
                    const double *target, double *residual_out);

/* Imaginary-time relaxation to a residual tolerance (the ground-state search
 * of Sec. 3.2 and Sec. 6, run until it has converged instead of for a fixed
 * number of steps).  Runs spgpe_step_imag in chunks of check_every steps, each
 * chunk ending with the discrete-map residual of its last step (defined as
 * for spgpe_step_imag), until every instance has residual <= tol or max_steps
 * steps have run.  An instance within tol is frozen (no longer stepped) while
 * the others go on.  dtau, norm_mode and target as for spgpe_step_imag.
 *
 * flags, a bitwise or of:
 *  SPGPE_RELAX_LADDER (complex128 contexts; ignored on complex64): relax a
 *   complex64 copy of the spinor with the same model first (the context's
 *   own complex64 twin, allocated on first use): rounded once, stepped in
 *   complex64 until every residual is <= max(tol, handoff), or, with
 *   handoff = 0, until each instance's residual has reached complex64's
 *   rounding floor (below 2^-18 / dtau) and improves by less than a fifth per
 *   chunk (an instance at the floor is stepped on until the last one gets
 *   there); then widened back into psi and relaxed in complex128 to tol.  The
 *   two stages share max_steps: the complex128 stage runs at most max_steps
 *   minus the steps the complex64 stage ran.  The rounding of every complex64 step
 *   also excites slowly relaxing modes that a smooth initial state leaves
 *   untouched, so the ladder pays off for initial states far from the ground
 *   state (random or vortex-seeded), and a hand-off residual well above the
 *   floor limits that noise.
 *  SPGPE_RELAX_GIVE_UP: also freeze an instance whose smallest residual so
 *   far has not halved in 40 chunks (a metastable state, or a relaxation far
 *   too slow for the budget); its residual stays above tol.
 *  SPGPE_RELAX_LAGGED: run the chunks with the lagged renormalisation of
 *   spgpe_step_imag (SPGPE_IMAG_LAGGED); the last step of every chunk stays
 *   exact, so the residuals compared with tol are those of the exact map.
 * handoff >= 0.  residual_out (host, nullable): ninst doubles, the last
 * residual of each instance.  steps_out (host, nullable): {steps run in
 * complex64 by the ladder, steps run in the context's precision}, counted
 * until the last instance of the stage was done.  Returns SPGPE_OK also when
 * max_steps ran out first (compare residual_out with tol).  Synchronises. */
enum { SPGPE_RELAX_LADDER = 1, SPGPE_RELAX_GIVE_UP = 2, SPGPE_RELAX_LAGGED = 4 };
int spgpe_relax(spgpe_ctx *ctx, void *psi, double dtau, double tol, int max_steps, int check_every,
                int norm_mode, const double *target, int flags, double handoff, double *residual_out,
                int *steps_out);

/* Autotuning of the pass schedule: for the grid of a single-size context, or
 * for every size class of a multi-size batch, time real-time steps S(dt) of
 * each schedule (variant v: bit 0 set = persistent row pass, in which each
 * warp or block streams its next rows into shared memory while it transforms
 * the current ones, else one row group per block; v >> 1 = column pass:
 * 0 one column tile per block, 1 persistent TMA pass, 2 warp-local TMA pass
 * with the 128-byte swizzle (complex64 grids with ny = 256 only)) on a
 * scratch copy of psi (psi itself is not changed), twice each, and keep the
 * fastest for all later calls (complex64 twins included).  choice_out (host,
 * nullable): the chosen variant per class (one entry for a single-size
 * context); ms_out (host, nullable): its time per step in milliseconds.
 * Synchronises. */
int spgpe_autotune(spgpe_ctx *ctx, const void *psi, double dt, int *choice_out, double *ms_out);

/* Energy functional whose variation is H Psi, per instance:
 * out[6*i .. 6*i+5] = {E_total, E_kinetic (incl. -kL kx sigma_z), E_trap,
 * E_detuning, E_Raman, E_interaction}, extensive (divide by the atom number
 * for per-particle values).  Kinetic part by Parseval on the 2D FFT.  FP64
 * accumulation; synchronises.  ENONFINITE if any sum is not finite. */
int spgpe_energy(spgpe_ctx *ctx, const void *psi, double *out);

/* Atom numbers per instance, out[2*i] = N_up, out[2*i+1] = N_dn, FP64
 * accumulation; synchronises.  ENONFINITE if a sum is not finite. */
int spgpe_norm(spgpe_ctx *ctx, const void *psi, double *out);

/* Observables of the spin-Hall ground states (Sec. 6), per instance:
 * out[4*i .. 4*i+3] = {s, n_up, n_dn, R99}.
 *  s: phase-separation parameter (Eq. 14), read as
 *     1 - sum rho_up rho_dn / sqrt(sum rho_up^2 sum rho_dn^2) over the grid
 *     (0 for proportional densities, 1 for disjoint ones).
 *  R99: radius of the circle about the trap centre (0, 0) that encloses 99 %
 *     of the total atom number (radii binned in widths min(dx, dy)/2; the
 *     upper edge of the first bin at which the cumulative number reaches 99 %).
 *  n_j: winding number of arg psi_j around that circle, counter-clockwise,
 *     from 4 max(nx, ny) equally spaced points with psi_j bilinearly
 *     interpolated on the periodic grid (phase steps wrapped into (-pi, pi],
 *     summed in FP64, divided by 2 pi and rounded); the circulation of
 *     Eq. 15 is 2 pi n_j (hbar = m = 1).
 * Synchronises.  ENONFINITE if a value is not finite (e.g. a zero spinor). */
int spgpe_observables(spgpe_ctx *ctx, const void *psi, double *out);

/* Annealing noise of the ground-state protocol (Sec. 6: the first
 * imaginary-time segment is perturbed now and then with Gaussian noise):
 * psi += sigma xi, xi complex standard normal (E|xi|^2 = 1), independent per
 * element.  Element e (component-major, then row-major) of global instance i
 * takes draws 2E and 2E + 1, E = i * 2 nx ny + e, of the counter-based
 * SplitMix64 stream `seed` (draw c = output function of seed + (c + 1)
 * 0x9E3779B97F4A7C15; Steele, Lea & Flood 2014), as uniforms u = (draw >> 11)
 * 2^-53, and xi = sqrt(-ln(1 - u1)) e^{2 pi i u2}.  The spinor is not
 * renormalised (the next imaginary-time step does that).  Stream-ordered;
 * a host spinor makes the call synchronous.  EINVAL for sigma < 0 or NaN. */
int spgpe_add_noise(spgpe_ctx *ctx, void *psi, double sigma, unsigned long long seed);

/* Wait for the context's stream and report an error recorded on the device
 * by an earlier asynchronous step (ENONFINITE, ETIMEOUT), clearing it. */
int spgpe_sync(spgpe_ctx *ctx);

/* Probe of the bounded-wait failure path of the streaming passes: one kernel
 * on the context's stream (the first size class of a multi-size context)
 * waits, for about `cycles` SM clock cycles, on a shared-memory barrier that
 * nothing completes, then records the timeout in the context's error flags
 * and exits with nothing in flight, as a pass does when a tile transfer
 * never lands.  Synchronises and returns what the next synchronising call
 * would: ETIMEOUT (the flag is cleared and the context stays usable), or
 * ECUDA if the launch failed.  EINVAL for cycles < 0. */
int spgpe_wait_probe(spgpe_ctx *ctx, long long cycles);

/* Comparator with the paper's structure (Sec. 4): the same S(dt) built from
 * cuFFT 2D transforms and separate elementwise kernels, several passes over
 * psi per step.  Kept for timing and as a second witness; real time only,
 * device psi only. */
int spgpe_cufft_step_real(spgpe_ctx *ctx, void *psi, double dt, int nsteps);

/* ---- Learned warm start: a Fourier neural operator (FNO) ----
 * Not part of the paper's method: a network (the Fourier neural operator of
 * Li et al., arXiv:2010.08895) trained on ground states this library computes,
 * whose output seeds the imaginary-time relaxation of Sec. 3.2 (which still
 * decides the result and its residual: spgpe_relax).  It maps input fields
 * a[batch][cin][n][n] to output fields out[batch][cout][n][n] (float32,
 * device memory, x fastest):
 *   v_0 = P a + p;  u_l = W_l v_l + w_l + S_l(v_l),  v_{l+1} = gelu(u_l)
 *   (l < layers - 1), v_layers = u_{layers-1};  out = Q2 gelu(Q1 v + q1) + q2,
 * gelu(x) = x Phi(x), and the spectral convolution S over the kept modes
 * kx = 0..modes-1, ky = 0..modes-1 and n-modes..n-1:
 *   vh = sum_{y,x} v exp(-2 pi i (kx x + ky y)/n);  oh[o] = sum_c R[ky][kx][o][c] vh[c];
 *   S(v) = Re sum g_kx oh exp(+2 pi i (kx x + ky y)/n) / n^2,  g_0 = 1, g_kx = 2.
 * Parameters are one float32 vector: P [width][cin], p [width]; per layer
 * W_l [width][width], w_l [width], R_l [2 modes][modes][width][width][2]
 * (real, imaginary); Q1 [hidden][width], q1 [hidden], Q2 [cout][hidden],
 * q2 [cout].  The products use the weights rounded to bfloat16 and
 * accumulate in float32; Adam updates the float32 masters.  The loss of a
 * batch is the mean relative squared error
 * sum_b ||out_b - target_b||^2 / ||target_b||^2 / batch.  n is a power of two
 * with 2 modes <= n <= 4096.  A model is not thread-safe; calls are
 * stream-ordered on cuda_stream and synchronise only where stated. */
typedef struct spgpe_fno spgpe_fno;

/* Allocate a model with seeded initial weights (matrices uniform in
 * +-1/sqrt(fan_in), biases zero, spectral weights uniform in [0, 1)/width^2).
 * EINVAL for non-positive or excessive sizes, ENOMEM/ECUDA on failure. */
int spgpe_fno_create(spgpe_fno **out, int cin, int cout, int width, int modes, int layers, int hidden,
                     unsigned long long seed, void *cuda_stream);
/* Number of float32 parameters. */
long spgpe_fno_num_params(const spgpe_fno *f);
/* Copy the float32 master parameters to / from the host (synchronises); set
 * also resets the Adam moments and step count. */
int spgpe_fno_get_params(spgpe_fno *f, float *host);
int spgpe_fno_set_params(spgpe_fno *f, const float *host);
/* out = FNO(a) for a batch of inputs (device pointers). */
int spgpe_fno_forward(spgpe_fno *f, const float *a, int batch, int n, float *out);
/* Forward pass into out, loss (host, nullable; synchronises) and the gradient
 * of the loss with respect to every parameter, copied to grad_host (host,
 * nullable, num_params floats; synchronises). */
int spgpe_fno_gradient(spgpe_fno *f, const float *a, const float *target, int batch, int n, float *out,
                       double *loss, float *grad_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * batch with learning rate lr; out receives the forward pass and loss (host,
 * nullable) the loss before the step. */
int spgpe_fno_train_step(spgpe_fno *f, const float *a, const float *target, int batch, int n, float *out,
                         double lr, double *loss);
void spgpe_fno_destroy(spgpe_fno *f);
const char *spgpe_fno_last_error(const spgpe_fno *f);

void spgpe_destroy(spgpe_ctx *ctx);
const char *spgpe_last_error(const spgpe_ctx *ctx);
int spgpe_version(void);

/* Introspection for benchmarks: number of kernel launches the last step call
 * issued (real time 2*nsteps + 1, imaginary time 3*nsteps + 1 with the exact
 * rescaling, 2*nsteps + 3 with SPGPE_IMAG_LAGGED and nsteps >= 2, both
 * without residual_out). */
int spgpe_last_launches(const spgpe_ctx *ctx);

/* Per-kernel timing for benchmarks.  While enabled (enable = 1), every fused
 * launch is bracketed by CUDA events recorded on the context's stream.
 * spgpe_timing synchronises and writes, for each kernel kind k in
 * [0, SPGPE_NKINDS), the launch count count_out[k] and the summed event time
 * ms_out[k] since timing was enabled, then restarts the accumulation.  Kinds:
 * 0 real row pass opening, 1 real row pass fused (step end + next start),
 * 2 real row pass closing, 3 real column pass, 4 imaginary row opening,
 * 5 imaginary row pass B (scale + R + FFT), 6 imaginary row pass A (IFFT + R +
 * norm partials), 7 imaginary rescale, 8 imaginary column pass, 9 imaginary
 * lagged row pass (IFFT + R + norm partials + predicted scale + R + FFT). */
#define SPGPE_NKINDS 10
int spgpe_set_timing(spgpe_ctx *ctx, int enable);
int spgpe_timing(spgpe_ctx *ctx, double *ms_out, int *count_out);

/* Microbenchmarks of this GPU's ceilings, for reading the measured kernel
 * times against (no counterpart in the paper; it only launches kernels on a
 * stream of its own, on the current device, and changes no device setting).
 * out (host, n_out >= SPGPE_PROBE_COUNT doubles) receives:
 *  out[0] FP32 fused multiply-add throughput, TFLOP/s (2 flop per fma);
 *  out[1] FP64 fused multiply-add throughput, TFLOP/s;
 *  out[2] sincosf throughput, 10^9 calls/s (arguments in [0, 1]);
 *  out[3] copy bandwidth over 512 MiB + 512 MiB, GB/s (bytes read + written);
 *  out[4 + k] read bandwidth, GB/s, over a working set of 16, 32, 64, 96, 128,
 *   160, 192, 256, 512 MiB for k = 0 .. 8, each read repeatedly (about 2 GiB
 *   per measurement): the drop between sizes marks the L2 capacity.
 * Each figure is one CUDA-event-timed launch after an untimed one.
 * Allocates 1 GiB of device memory for the duration of the call and
 * synchronises.  EINVAL for out NULL or n_out too small; ENOMEM / ECUDA. */
#define SPGPE_PROBE_NSIZES 9
#define SPGPE_PROBE_COUNT (4 + SPGPE_PROBE_NSIZES)
int spgpe_probe_ceilings(double *out, int n_out);

/* Atom numbers of a spinor batch without allocating any memory (the paper has
 * no counterpart: this serves callers that cannot call cudaMalloc, such as
 * host applications or plugins that hand out all device memory from their own
 * pool, or that run under a fixed device-memory budget where a library may not
 * allocate).  No context is needed and the call allocates nothing, on the
 * device or the host: the partial sums live in a 256 KiB array of device
 * memory that is part of the library's device code.  The CUDA runtime
 * reserves that array on a GPU when it loads the library's module there (with
 * lazy module loading, possibly during the first call), and the GPU keeps it
 * until the process exits.  psi is the caller's device buffer [ninst][2][ny][nx] complex of the
 * given dtype (SPGPE_C64 or SPGPE_C128) over [-xmax, xmax) x [-ymax, ymax);
 * out is a host array of 2*ninst doubles receiving {N_up, N_dn} per instance
 * (dx dy sum |psi_j|^2, FP64 accumulation).  Runs on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream) and synchronises it.
 * The first call on a device looks up the device address of the array, so
 * make that first call before any stream capture.  All calls share the one
 * array: calls that overlap on the GPU (from several streams or threads) race
 * and must be serialised by the caller.  Returns EINVAL for NULL pointers,
 * sizes below one, nx*ny above 2^30, a bad dtype or extent, or ninst above
 * 252 (the capacity of the array); ECUDA when a CUDA call fails; ENONFINITE if
 * a sum is not finite. */
int spgpe_norm_noalloc(const void *psi, int nx, int ny, int ninst, double xmax,
                       double ymax, int dtype, void *cuda_stream, double *out);

#ifdef __cplusplus
}
#endif
#endif /* SPGPE_H */
