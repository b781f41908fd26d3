// Plain FP64 reference ("oracle") for the Strang time-splitting spectral (TSSP)
// step of the two-component quasi-2D Gross-Pitaevskii equation of
// arXiv:2010.15069 (Smith, Cooke, LeBlanc, "GPU-accelerated solutions of the
// NLSE for simulating 2D spinor BECs").
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct CPU
// definition that the CUDA library is checked against.  Only the tests, the
// package's smoke check and the benchmark's CPU-baseline leg may load it.  It
// shares no code, header, table or constant with the CUDA path.
//
// Conventions (oscillator units, hbar = m = omega_perp = 1):
//  * Grid (Sec. 3.2): x_i = -xmax + i*dx, dx = 2*xmax/nx, i = 0..nx-1 (periodic,
//    +xmax excluded); kx = 2*pi*fftfreq(nx, dx), Nyquist carried as -pi/dx.
//    Same for y.  Arrays are [ny][nx] row-major, x fastest; a spinor is
//    [2][ny][nx] (component up first), complex interleaved (re, im).
//  * Hamiltonian: signs of Eq. 3 with hbar = m = 1,
//      H = diag(T_up, T_dn)(k) + V 1 + (delta/2) sigma_z + (Omega/2) sigma_x
//          + diag(g11 rho_up + g12 rho_dn, g22 rho_dn + g12 rho_up),
//      T_up(k) = k^2/2 - kL*kx,  T_dn(k) = k^2/2 + kL*kx.
//    Eqs. 4-8 print H(1) with the opposite overall sign together with
//    exp(+i H dt) (Eq. 13); the two sign flips cancel in real time up to time
//    reversal, and imaginary time (dt -> -i dtau) gives exp(-H dtau) either way.
//    This file uses i dPsi/dt = H Psi: real time exp(-i H dt), imaginary time
//    exp(-H dtau).
//  * Forward transform sum_x e^{-i k x} (unnormalised), inverse sum_k e^{+i k x}
//    divided by nx*ny (Sec. 3.2: H(1) is diagonal in k space, Laplacian -> -k^2).
//  * Sub-operators for a substep tau (Eq. 13 with the operator split of
//    Sec. 3.2):
//      D(tau): psi_up *= exp(-i tau (V + delta/2 + g11 rho_up + g12 rho_dn)),
//              psi_dn *= exp(-i tau (V - delta/2 + g22 rho_dn + g12 rho_up)),
//              densities taken at substep entry (imaginary: exp(-tau (...))).
//      X(tau): exp(-i tau Omega sigma_x / 2) (imaginary: exp(-tau Omega sigma_x/2)).
//      K(tau): psi_hat_j *= exp(-i tau T_j(k)) (imaginary: exp(-tau T_j(k))).
//      R(tau) = X(tau/2) D(tau) X(tau/2)   (second-order split of the
//               real-space operators U(2), U(3), U(4), Sec. 3.2).
//    One step: S(dt) = R(dt/2) . F^-1 K(dt) F . R(dt/2): four 2D FFTs per
//    step (two components, forward and inverse), as Sec. 3.2 counts.
//  * Imaginary time: after each S(dtau) the spinor is rescaled to the target
//    atom number (Sec. 3.2), either the total (mode 0) or per component
//    (mode 1).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

namespace {

using cd = std::complex<double>;
const double kPi = 3.14159265358979323846264338327950288;

// ---- own iterative radix-2 Cooley-Tukey FFT (Sec. 3.2 "FFT to k space") ----

// In-place length-n transform of a[0], a[stride], ..., a[(n-1)*stride].
// sign = -1: forward sum_j a_j e^{-2 pi i jk/n}; sign = +1: the same with
// e^{+...}.  Neither direction is normalised.  n must be a power of two.
void fft1d(cd *a, int n, long stride, int sign, const std::vector<cd> &w) {
  // w[m] = exp(sign * 2 pi i m / n), m < n/2.
  for (int i = 1, j = 0; i < n; ++i) {  // bit-reversal permutation
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i * stride], a[j * stride]);
  }
  for (int len = 2; len <= n; len <<= 1) {  // butterflies, span len/2
    const int half = len / 2, step = n / len;
    for (int i = 0; i < n; i += len)
      for (int k = 0; k < half; ++k) {
        const cd u = a[(i + k) * stride];
        const cd v = a[(i + k + half) * stride] * w[k * step];
        a[(i + k) * stride] = u + v;
        a[(i + k + half) * stride] = u - v;
      }
  }
}

std::vector<cd> roots(int n, int sign) {
  std::vector<cd> w(n / 2 > 0 ? n / 2 : 1);
  for (int m = 0; m < n / 2; ++m) {
    const double t = sign * 2.0 * kPi * m / n;
    w[m] = cd(std::cos(t), std::sin(t));
  }
  return w;
}

// 2D transform of one [ny][nx] plane: every row, then every column.
void fft2d(cd *p, int nx, int ny, int sign) {
  const std::vector<cd> wx = roots(nx, sign), wy = roots(ny, sign);
  for (int iy = 0; iy < ny; ++iy) fft1d(p + (long)iy * nx, nx, 1, sign, wx);
  for (int ix = 0; ix < nx; ++ix) fft1d(p + ix, ny, nx, sign, wy);
}

}  // namespace

extern "C" {

// Model of the pseudospinor NLSE (Eqs. 3-8).  Potential arrays are [ny][nx]
// FP64, NULL meaning identically zero.
struct orc_model {
  int nx, ny;
  double xmax, ymax;
  const double *V;
  const double *delta;
  const double *Omega;
  double g11, g22, g12, kL;
};

}  // extern "C"

namespace {

double dx_of(const orc_model *m) { return 2.0 * m->xmax / m->nx; }
double dy_of(const orc_model *m) { return 2.0 * m->ymax / m->ny; }

// Angular wavenumber of FFT bin i for length n and spacing d (numpy fftfreq
// convention times 2 pi: bins n/2..n-1 are negative, Nyquist negative).
double kbin(int i, int n, double d) {
  const int f = (i < n / 2) ? i : i - n;
  return 2.0 * kPi * f / (n * d);
}

double at(const double *a, long i) { return a ? a[i] : 0.0; }

// D(tau), Sec. 3.2 / Eq. 7 plus the diagonal part of Eq. 6.
void apply_D(const orc_model *m, cd *up, cd *dn, double tau, int imag) {
  const long n = (long)m->nx * m->ny;
  for (long i = 0; i < n; ++i) {
    const double ru = std::norm(up[i]), rd = std::norm(dn[i]);
    const double v = at(m->V, i), d = at(m->delta, i);
    const double eu = v + 0.5 * d + m->g11 * ru + m->g12 * rd;
    const double ed = v - 0.5 * d + m->g22 * rd + m->g12 * ru;
    if (imag) {
      up[i] *= std::exp(-tau * eu);
      dn[i] *= std::exp(-tau * ed);
    } else {
      up[i] *= std::polar(1.0, -tau * eu);
      dn[i] *= std::polar(1.0, -tau * ed);
    }
  }
}

// X(tau) = exp(-i tau Omega sigma_x / 2), Eq. 8 (imaginary: exp(-tau Omega sigma_x/2)).
void apply_X(const orc_model *m, cd *up, cd *dn, double tau, int imag) {
  if (!m->Omega) return;
  const long n = (long)m->nx * m->ny;
  for (long i = 0; i < n; ++i) {
    const double a = 0.5 * m->Omega[i] * tau;
    const cd u = up[i], d = dn[i];
    if (imag) {
      const double c = std::cosh(a), s = std::sinh(a);
      up[i] = c * u - s * d;
      dn[i] = -s * u + c * d;
    } else {
      const double c = std::cos(a), s = std::sin(a);
      const cd mis(0.0, -s);
      up[i] = c * u + mis * d;
      dn[i] = mis * u + c * d;
    }
  }
}

void apply_R(const orc_model *m, cd *up, cd *dn, double tau, int imag) {
  apply_X(m, up, dn, 0.5 * tau, imag);
  apply_D(m, up, dn, tau, imag);
  apply_X(m, up, dn, 0.5 * tau, imag);
}

// K(tau) on transformed planes, Eq. 5 with T_j(k) of Eq. 3; also divides by
// nx*ny, the normalisation of the inverse transform that follows.
void apply_K(const orc_model *m, cd *uh, cd *dh, double tau, int imag) {
  const double dx = dx_of(m), dy = dy_of(m), inv = 1.0 / ((double)m->nx * m->ny);
  for (int iy = 0; iy < m->ny; ++iy) {
    const double ky = kbin(iy, m->ny, dy);
    for (int ix = 0; ix < m->nx; ++ix) {
      const double kx = kbin(ix, m->nx, dx);
      const double k2 = 0.5 * (kx * kx + ky * ky);
      const double tu = k2 - m->kL * kx, td = k2 + m->kL * kx;
      const long i = (long)iy * m->nx + ix;
      if (imag) {
        uh[i] *= inv * std::exp(-tau * tu);
        dh[i] *= inv * std::exp(-tau * td);
      } else {
        uh[i] *= inv * std::polar(1.0, -tau * tu);
        dh[i] *= inv * std::polar(1.0, -tau * td);
      }
    }
  }
}

void norms(const orc_model *m, const cd *up, const cd *dn, double out[2]) {
  const long n = (long)m->nx * m->ny;
  const double w = dx_of(m) * dy_of(m);
  double su = 0.0, sd = 0.0;
  for (long i = 0; i < n; ++i) {
    su += std::norm(up[i]);
    sd += std::norm(dn[i]);
  }
  out[0] = w * su;
  out[1] = w * sd;
}

}  // namespace

extern "C" {

// 2D FFT of one plane in place (test hook for the FFT pins).
// sign -1 forward, +1 inverse; unnormalised in both directions.
void orc_fft2(int nx, int ny, double *plane, int sign) {
  fft2d(reinterpret_cast<cd *>(plane), nx, ny, sign);
}

// Apply one named sub-operator to a spinor (test hook).
// which: 0 = D(tau), 1 = X(tau), 2 = R(tau), 3 = F^-1 K(tau) F.
void orc_apply(const orc_model *m, double *psi, double tau, int imag, int which) {
  const long n = (long)m->nx * m->ny;
  cd *up = reinterpret_cast<cd *>(psi), *dn = up + n;
  switch (which) {
    case 0: apply_D(m, up, dn, tau, imag); break;
    case 1: apply_X(m, up, dn, tau, imag); break;
    case 2: apply_R(m, up, dn, tau, imag); break;
    case 3:
      fft2d(up, m->nx, m->ny, -1);
      fft2d(dn, m->nx, m->ny, -1);
      apply_K(m, up, dn, tau, imag);
      fft2d(up, m->nx, m->ny, +1);
      fft2d(dn, m->nx, m->ny, +1);
      break;
    default: break;
  }
}

// nsteps Strang steps S(dt) (Sec. 3.2, Fig. 1 loop), in place on psi.
// imag = 1: imaginary time, rescaling after every step to target[] (mode 0:
// total atom number target[0] + target[1]; mode 1: per component).
// residual_out (nullable, imaginary time): discrete-map residual of the last
// step, ||Psi_{n+1} - Psi_n|| / (dtau ||Psi_n||), grid-weighted L2 over both
// components, where Psi_n is the (normalised) state entering the last step.
void orc_step(const orc_model *m, double *psi, double dt, int nsteps, int imag,
              int norm_mode, const double *target, double *residual_out) {
  const long n = (long)m->nx * m->ny;
  cd *up = reinterpret_cast<cd *>(psi), *dn = up + n;
  std::vector<cd> prev;
  for (int s = 0; s < nsteps; ++s) {
    if (residual_out && s == nsteps - 1) prev.assign(up, up + 2 * n);
    apply_R(m, up, dn, 0.5 * dt, imag);
    fft2d(up, m->nx, m->ny, -1);
    fft2d(dn, m->nx, m->ny, -1);
    apply_K(m, up, dn, dt, imag);
    fft2d(up, m->nx, m->ny, +1);
    fft2d(dn, m->nx, m->ny, +1);
    apply_R(m, up, dn, 0.5 * dt, imag);
    if (imag) {
      double nn[2];
      norms(m, up, dn, nn);
      if (norm_mode == 1) {
        const double cu = std::sqrt(target[0] / nn[0]);
        const double cdn = std::sqrt(target[1] / nn[1]);
        for (long i = 0; i < n; ++i) { up[i] *= cu; dn[i] *= cdn; }
      } else {
        const double c = std::sqrt((target[0] + target[1]) / (nn[0] + nn[1]));
        for (long i = 0; i < n; ++i) { up[i] *= c; dn[i] *= c; }
      }
    }
  }
  if (residual_out) {
    if (nsteps <= 0) { *residual_out = NAN; return; }
    double num = 0.0, den = 0.0;
    for (long i = 0; i < 2 * n; ++i) {
      num += std::norm(up[i] - prev[i]);
      den += std::norm(prev[i]);
    }
    *residual_out = std::sqrt(num / den) / dt;
  }
}

// Atom numbers {N_up, N_dn} = dx dy sum |psi_j|^2.
void orc_norm(const orc_model *m, const double *psi, double out[2]) {
  const long n = (long)m->nx * m->ny;
  const cd *up = reinterpret_cast<const cd *>(psi);
  norms(m, up, up + n, out);
}

// Gross-Pitaevskii energy functional whose variation dE/dPsi* is H Psi:
// out = {E_total, E_kinetic (incl. the kL kx sigma_z term), E_trap,
// E_detuning, E_Raman, E_interaction}, extensive (not divided by N).
void orc_energy(const orc_model *m, const double *psi, double out[6]) {
  const int nx = m->nx, ny = m->ny;
  const long n = (long)nx * ny;
  const double dx = dx_of(m), dy = dy_of(m), w = dx * dy;
  const cd *up = reinterpret_cast<const cd *>(psi), *dn = up + n;
  std::vector<cd> uh(up, up + n), dh(dn, dn + n);
  fft2d(uh.data(), nx, ny, -1);
  fft2d(dh.data(), nx, ny, -1);
  double ekin = 0.0;
  for (int iy = 0; iy < ny; ++iy) {
    const double ky = kbin(iy, ny, dy);
    for (int ix = 0; ix < nx; ++ix) {
      const double kx = kbin(ix, nx, dx);
      const double k2 = 0.5 * (kx * kx + ky * ky);
      const long i = (long)iy * nx + ix;
      ekin += (k2 - m->kL * kx) * std::norm(uh[i]) + (k2 + m->kL * kx) * std::norm(dh[i]);
    }
  }
  ekin *= w / (double)n;  // Parseval: sum_r |psi|^2 = (1/N) sum_k |psi_hat|^2
  double etrap = 0.0, edet = 0.0, eram = 0.0, eint = 0.0;
  for (long i = 0; i < n; ++i) {
    const double ru = std::norm(up[i]), rd = std::norm(dn[i]);
    etrap += at(m->V, i) * (ru + rd);
    edet += 0.5 * at(m->delta, i) * (ru - rd);
    eram += at(m->Omega, i) * std::real(std::conj(up[i]) * dn[i]);
    eint += 0.5 * m->g11 * ru * ru + 0.5 * m->g22 * rd * rd + m->g12 * ru * rd;
  }
  out[1] = ekin;
  out[2] = w * etrap;
  out[3] = w * edet;
  out[4] = w * eram;
  out[5] = w * eint;
  out[0] = out[1] + out[2] + out[3] + out[4] + out[5];
}

// ---- observables of the spin-Hall ground states (Sec. 6) ----

// Phase-separation parameter (Eq. 14) and circulation (Eq. 15) of one spinor:
// out = {s, n_up, n_dn, R99}.
//  * s = 1 - sum rho_up rho_dn / sqrt(sum rho_up^2 sum rho_dn^2), sums over
//    the grid.  Eq. 14 prints the sum over r outside the bracket of averages;
//    read (as in the work it cites, and so that s lies in [0, 1]: 0 for
//    rho_up proportional to rho_dn, 1 for disjoint densities) as the averages
//    being those sums.
//  * R99: the radius of the circle about the trap centre (0, 0) that encloses
//    99 % of the total atom number: radii binned in widths h = min(dx, dy)/2,
//    R99 = upper edge of the first bin at which the cumulative atom number
//    reaches 0.99 of the total.
//  * n_j: winding number of phi_j = arg psi_j around that circle,
//    counter-clockwise, from `npts` equally spaced points (angles 2 pi k /
//    npts), psi_j bilinearly interpolated on the periodic grid; the phase
//    steps wrapped into (-pi, pi] are summed and the sum / 2 pi rounded.  The
//    circulation of Eq. 15 is 2 pi n_j (hbar = m = 1).
void orc_observables(const orc_model *m, const double *psi, int npts, double out[4]) {
  const int nx = m->nx, ny = m->ny;
  const long n = (long)nx * ny;
  const double dx = dx_of(m), dy = dy_of(m);
  const cd *up = reinterpret_cast<const cd *>(psi), *dn = up + n;
  double a = 0.0, b = 0.0, c = 0.0, tot = 0.0;
  for (long i = 0; i < n; ++i) {
    const double ru = std::norm(up[i]), rd = std::norm(dn[i]);
    a += ru * rd;
    b += ru * ru;
    c += rd * rd;
    tot += ru + rd;
  }
  out[0] = 1.0 - a / std::sqrt(b * c);
  // radial distribution of the total density
  const double h = 0.5 * std::min(dx, dy);
  const double rmax = std::sqrt(m->xmax * m->xmax + m->ymax * m->ymax);
  const int nb = (int)(rmax / h) + 2;
  std::vector<double> hist(nb, 0.0);
  for (int iy = 0; iy < ny; ++iy)
    for (int ix = 0; ix < nx; ++ix) {
      const double x = -m->xmax + ix * dx, y = -m->ymax + iy * dy;
      const long i = (long)iy * nx + ix;
      const int bin = std::min(nb - 1, (int)(std::sqrt(x * x + y * y) / h));
      hist[bin] += std::norm(up[i]) + std::norm(dn[i]);
    }
  double cum = 0.0, R = (nb) * h;
  for (int k = 0; k < nb; ++k) {
    cum += hist[k];
    if (cum >= 0.99 * tot) {
      R = (k + 1) * h;
      break;
    }
  }
  out[3] = R;
  // winding of each component around the circle of radius R
  auto interp = [&](const cd *f, double x, double y) {
    const double u = (x + m->xmax) / dx, v = (y + m->ymax) / dy;
    const double fu = u - std::floor(u), fv = v - std::floor(v);
    const long i0 = (((long)std::floor(u)) % nx + nx) % nx, j0 = (((long)std::floor(v)) % ny + ny) % ny;
    const long i1 = (i0 + 1) % nx, j1 = (j0 + 1) % ny;
    return (1 - fu) * (1 - fv) * f[j0 * nx + i0] + fu * (1 - fv) * f[j0 * nx + i1] +
           (1 - fu) * fv * f[j1 * nx + i0] + fu * fv * f[j1 * nx + i1];
  };
  for (int j = 0; j < 2; ++j) {
    const cd *f = j == 0 ? up : dn;
    double total = 0.0;
    double prev = std::arg(interp(f, R, 0.0));
    for (int k = 1; k <= npts; ++k) {
      const double th = 2.0 * kPi * (double)(k % npts) / npts;
      const double ph = std::arg(interp(f, R * std::cos(th), R * std::sin(th)));
      double d = ph - prev;
      while (d > kPi) d -= 2.0 * kPi;
      while (d <= -kPi) d += 2.0 * kPi;
      total += d;
      prev = ph;
    }
    out[1 + j] = std::round(total / (2.0 * kPi));
  }
}

// ---- annealing noise (Sec. 6: the first imaginary-time segment is
// periodically perturbed with Gaussian noise) ----

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based generator:
// draw c of stream `seed` is the output function applied to
// seed + (c + 1) * 0x9E3779B97F4A7C15.
unsigned long long orc_splitmix64(unsigned long long seed, unsigned long long c) {
  unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// psi += sigma xi with xi complex standard normal (E|xi|^2 = 1), independent
// per element: element e (component-major, then row-major) of instance `inst`
// takes the draws c = 2 E + 0 and 2 E + 1, E = inst * 2 nx ny + e, as
// uniforms u = (draw >> 11) 2^-53, and xi = sqrt(-ln(1 - u1)) e^{2 pi i u2}
// (Box-Muller in polar form).
void orc_add_noise(const orc_model *m, double *psi, double sigma, unsigned long long seed, long inst) {
  const long n2 = 2L * m->nx * m->ny;
  cd *p = reinterpret_cast<cd *>(psi);
  for (long e = 0; e < n2; ++e) {
    const unsigned long long E = (unsigned long long)(inst * n2 + e);
    const double u1 = (double)(orc_splitmix64(seed, 2 * E) >> 11) * 0x1.0p-53;
    const double u2 = (double)(orc_splitmix64(seed, 2 * E + 1) >> 11) * 0x1.0p-53;
    const double r = std::sqrt(-std::log(1.0 - u1));
    p[e] += sigma * r * cd(std::cos(2.0 * kPi * u2), std::sin(2.0 * kPi * u2));
  }
}

}  // extern "C"
