"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle's tests.

This module only *makes inputs*: grids of coordinates, trap/detuning/Raman
profiles, initial spinors and parameter draws.  It holds none of the method's
arithmetic (no evolution operator, FFT step or normalisation rule of the TSSP
scheme), so the CUDA path and the oracle can both consume its arrays without
sharing any of the computation they are compared on.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output k (k = 1, 2, ...) of the
stream with seed s is mix(s + k * 0x9E3779B97F4A7C15) with the published
64-bit finaliser, and u = (z >> 11) * 2^-53 is uniform in [0, 1).  Draws are
taken component-major, then row-major (y outer, x inner).

Units are oscillator units of the paper's example (Sec. 6): length
a0 = sqrt(hbar / m omega_perp), energy hbar omega_perp.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+n of the SplitMix64 stream with this seed (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from SplitMix64 (53-bit mantissa)."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass(frozen=True)
class Grid:
    """Uniform periodic grid x_i = -xmax + i dx, dx = 2 xmax / nx (Sec. 3.2)."""
    nx: int
    ny: int
    xmax: float
    ymax: float

    @property
    def dx(self) -> float:
        return 2.0 * self.xmax / self.nx

    @property
    def dy(self) -> float:
        return 2.0 * self.ymax / self.ny

    @property
    def x(self) -> np.ndarray:
        return -self.xmax + self.dx * np.arange(self.nx)

    @property
    def y(self) -> np.ndarray:
        return -self.ymax + self.dy * np.arange(self.ny)

    def mesh(self):
        """(X, Y) coordinate arrays of shape (ny, nx)."""
        return np.meshgrid(self.x, self.y, indexing="xy")


# ---------------------------------------------------------------- potentials

def harmonic_1d(g: Grid, omega: float = 1.0):
    """Separable pieces (Vx, Vy) of V = omega^2 (x^2 + y^2) / 2."""
    return 0.5 * omega ** 2 * g.x ** 2, 0.5 * omega ** 2 * g.y ** 2


def harmonic(g: Grid, omega: float = 1.0) -> np.ndarray:
    vx, vy = harmonic_1d(g, omega)
    return vy[:, None] + vx[None, :]


def gradient_y(g: Grid, slope: float) -> np.ndarray:
    """delta(x, y) = slope * y as a (ny, nx) array."""
    return np.broadcast_to(slope * g.y[:, None], (g.ny, g.nx)).copy()


def constant(g: Grid, value: float) -> np.ndarray:
    return np.full((g.ny, g.nx), float(value))


def raman_profile_y(g: Grid, E_L: float) -> np.ndarray:
    """Omega(y) = E_L sqrt(8 y - y^2) where real, 0 elsewhere (Eq. 12), as (ny,)."""
    y = g.y
    return E_L * np.sqrt(np.clip(8.0 * y - y * y, 0.0, None))


# ---------------------------------------------------------- initial spinors

def _normalise(psi: np.ndarray, g: Grid, target) -> np.ndarray:
    w = g.dx * g.dy
    for j in range(2):
        n = w * np.sum(np.abs(psi[j]) ** 2)
        if n > 0 and target[j] > 0:
            psi[j] *= math.sqrt(target[j] / n)
    return psi


def gaussian_spinor(g: Grid, width: float = 1.0, noise: float = 1e-3, seed: int = 0,
                    target=(0.5, 0.5), center=(0.0, 0.0), momentum=(0.0, 0.0)) -> np.ndarray:
    """psi_j = exp(-r^2 / (2 w^2)) exp(i k0.r) exp(i phi_j), phi ~ U[-noise, noise].

    Returns complex128 (2, ny, nx), each component scaled to atom number target[j].
    """
    X, Y = g.mesh()
    env = np.exp(-((X - center[0]) ** 2 + (Y - center[1]) ** 2) / (2.0 * width ** 2))
    env = env * np.exp(1j * (momentum[0] * X + momentum[1] * Y))
    phi = noise * (2.0 * uniform01(seed, 2 * g.nx * g.ny) - 1.0)
    psi = env[None, :, :] * np.exp(1j * phi.reshape(2, g.ny, g.nx))
    return _normalise(psi.astype(np.complex128), g, target)


def vortex_spinor(g: Grid, n_vortices: int = 50, radius: float = 5.0, seed: int = 2,
                  target=(0.5, 0.5)) -> np.ndarray:
    """Gaussian envelope of width `radius` seeded with randomly placed vortices.

    Vortex centres are uniform in the disc of the given radius (r = R sqrt(u1),
    theta = 2 pi u2); the up component winds +1 around each, the down
    component -1 (the paper's spin-dependent seeding, Sec. 6).
    """
    u = uniform01(seed, 2 * n_vortices)
    r = radius * np.sqrt(u[0::2])
    th = 2.0 * math.pi * u[1::2]
    xv, yv = r * np.cos(th), r * np.sin(th)
    X, Y = g.mesh()
    phase = np.zeros_like(X)
    for a, b in zip(xv, yv):
        phase += np.arctan2(Y - b, X - a)
    env = np.exp(-(X ** 2 + Y ** 2) / (2.0 * radius ** 2))
    psi = np.stack([env * np.exp(1j * phase), env * np.exp(-1j * phase)]).astype(np.complex128)
    return _normalise(psi, g, target)


def upsample_spectral(psi: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Band-limited interpolation of a (2, ny0, nx0) spinor onto (2, ny, nx) by
    zero-padding its discrete spectrum (same box); the atom number is kept."""
    c, ny0, nx0 = psi.shape
    out = np.zeros((c, ny, nx), dtype=np.complex128)
    for j in range(c):
        s = np.fft.fftshift(np.fft.fft2(psi[j]))
        big = np.zeros((ny, nx), dtype=np.complex128)
        oy, ox = (ny - ny0) // 2, (nx - nx0) // 2
        big[oy:oy + ny0, ox:ox + nx0] = s
        out[j] = np.fft.ifft2(np.fft.ifftshift(big)) * (nx * ny) / (nx0 * ny0)
    return out


# ------------------------------------------------------------ configurations

@dataclass
class Problem:
    """One instance of the model of Eqs. 3-8 on a grid, with its potentials."""
    grid: Grid
    V: np.ndarray
    delta: np.ndarray | None
    Omega: np.ndarray | None
    g11: float
    g22: float
    g12: float
    kL: float
    separable: dict = field(default_factory=dict)  # 1D pieces when the profiles are sums


def problem(nx, ny, xmax, ymax, omega=1.0, Omega=0.0, delta_slope=0.0,
            g11=0.0, g22=0.0, g12=0.0, kL=0.0) -> Problem:
    """Harmonic trap, uniform Raman coupling, linear detuning delta = slope * y."""
    g = Grid(nx, ny, xmax, ymax)
    vx, vy = harmonic_1d(g, omega)
    sep = dict(Vx=vx, Vy=vy, delta_x=None, delta_y=(delta_slope * g.y if delta_slope else None),
               Omega_x=None, Omega_y=(np.full(ny, float(Omega)) if Omega else None))
    return Problem(g, harmonic(g, omega),
                   gradient_y(g, delta_slope) if delta_slope else None,
                   constant(g, Omega) if Omega else None,
                   g11, g22, g12, kL, sep)


def config0() -> Problem:
    """64^2, box [-10,10]^2, harmonic trap, g11 = g22 = 100, g12 = 95, no coupling."""
    return problem(64, 64, 10.0, 10.0, g11=100.0, g22=100.0, g12=95.0)


def config1(n: int = 256) -> Problem:
    """256^2, box [-10,10]^2, Omega = 2, delta = 0.5 y, kL = 1, g11 = g22 = g12 = 200."""
    return problem(n, n, 10.0, 10.0, Omega=2.0, delta_slope=0.5, g11=200.0, g22=200.0,
                   g12=200.0, kL=1.0)


def config2(g12: float = 1000.0, n: int = 1024) -> Problem:
    """1024^2, box [-24,24]^2, Omega = 4, delta = 0.2 y, kL = 2, g = 1000, g12 as given."""
    return problem(n, n, 24.0, 24.0, Omega=4.0, delta_slope=0.2, g11=1000.0, g22=1000.0,
                   g12=g12, kL=2.0)


def sweep_params(n_inst: int, seed: int = 3):
    """Per-instance (g, g12/g, Omega, delta slope) draws of the batched sweep:
    g log-uniform in [50, 2000], g12/g ~ U[0.8, 1.2], Omega ~ U[0, 6],
    delta slope ~ U[0, 1]; instance i draws its four numbers in that order."""
    u = uniform01(seed, 4 * n_inst).reshape(n_inst, 4)
    g = np.exp(np.log(50.0) + u[:, 0] * (np.log(2000.0) - np.log(50.0)))
    return [dict(g=float(g[i]), g12=float(g[i] * (0.8 + 0.4 * u[i, 1])),
                 Omega=float(6.0 * u[i, 2]), delta_slope=float(u[i, 3])) for i in range(n_inst)]
