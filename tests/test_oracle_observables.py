"""Pins of the oracle's Sec. 6 observables and annealing noise (no GPU).

Phase separation (Eq. 14): exact limits and the closed form for displaced
Gaussians.  Circulation (Eq. 15): exact winding numbers of (x +- i y)^m
states and of vortices inside / outside the 99 % contour; the contour radius
against the Gaussian closed form.  Noise: the published first SplitMix64
output, agreement with the package's own SplitMix64, and the statistics of a
complex standard normal.
"""
import math

import numpy as np
import pytest

from paper_2010_15069_gb300 import inputs


def model(orc, n=128, L=8.0):
    return orc.Model(n, n, L, L)


def mesh(m):
    g = inputs.Grid(m.nx, m.ny, m.xmax, m.ymax)
    return g.mesh()


def test_phase_separation_limits(orc):
    m = model(orc)
    X, Y = mesh(m)
    f = np.exp(-(X ** 2 + Y ** 2) / 2)
    assert abs(m.observables(np.stack([f, f]))[0]) < 1e-14
    assert abs(m.observables(np.stack([f, 0.3j * f]))[0]) < 1e-14     # proportional densities
    up, dn = np.where(X < 0, f, 0), np.where(X >= 0, f, 0)             # disjoint supports
    assert m.observables(np.stack([up, dn]).astype(complex))[0] == 1.0


@pytest.mark.parametrize("a", [0.25, 0.7, 1.3])
def test_phase_separation_of_displaced_gaussians(orc, a):
    """rho_j = exp(-((x -+ a)^2 + y^2)): the overlap ratio is exp(-2 a^2)."""
    m = model(orc, 128, 8.0)
    X, Y = mesh(m)
    up = np.exp(-((X - a) ** 2 + Y ** 2) / 2)
    dn = np.exp(-((X + a) ** 2 + Y ** 2) / 2)
    s = m.observables(np.stack([up, dn]).astype(complex))[0]
    assert abs(s - (1 - math.exp(-2 * a * a))) < 1e-12


@pytest.mark.parametrize("mu,md", [(1, -1), (2, 0), (-3, 2), (0, 0)])
def test_winding_numbers_of_vortex_states(orc, mu, md):
    m = model(orc)
    X, Y = mesh(m)
    env = np.exp(-(X ** 2 + Y ** 2) / 2)

    def vort(k):
        z = X + 1j * np.sign(k) * Y
        return env * z ** abs(k) if k else env.astype(complex)
    o = m.observables(np.stack([vort(mu), vort(md)]))
    assert (o[1], o[2]) == (mu, md)


def test_only_vortices_inside_the_contour_count(orc):
    m = model(orc, 128, 8.0)
    X, Y = mesh(m)
    env = np.exp(-(X ** 2 + Y ** 2) / 4)                      # rho = exp(-r^2/2): R99 = 2 sqrt(ln 10) = 3.03

    def core(x0, y0, s):                                     # unit-modulus vortex of sign s away from its core
        z = (X - x0) + 1j * s * (Y - y0)
        return z / np.sqrt(np.abs(z) ** 2 + 0.25)
    inside = env * core(0.6, -0.4, 1)
    outside = env * core(6.0, 0.5, 1) * core(-0.3, 0.2, -1)
    o = m.observables(np.stack([inside, outside]))
    assert 2.7 < o[3] < 3.4
    assert (o[1], o[2]) == (1, -1)


@pytest.mark.parametrize("w", [0.8, 1.5, 2.5])
def test_contour_radius_encloses_99_percent(orc, w):
    """rho = exp(-r^2 / w^2): the fraction inside R is 1 - exp(-R^2 / w^2)."""
    m = model(orc, 256, 10.0)
    X, Y = mesh(m)
    f = np.exp(-(X ** 2 + Y ** 2) / (2 * w * w))
    R = m.observables(np.stack([f, f]).astype(complex))[3]
    # one grid spacing: half for the bin width, half for the lattice of radii
    assert abs(R - w * math.sqrt(math.log(100.0))) <= m.dx


def test_splitmix64_published_value_and_package_generator(orc):
    # first output of SplitMix64 seeded with 0 (Steele, Lea & Flood)
    assert orc.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    ref = inputs.splitmix64(12345, 10)
    assert [orc.splitmix64(12345, c) for c in range(10)] == [int(v) for v in ref]


def test_noise_statistics_and_reproducibility(orc):
    m = model(orc, 64, 4.0)
    z = np.zeros((2, 64, 64), complex)
    a = m.add_noise(z, 0.1, seed=7)
    b = m.add_noise(z, 0.1, seed=7)
    c = m.add_noise(z, 0.1, seed=7, inst=1)
    assert np.array_equal(a, b) and not np.allclose(a, c)
    for xi in (a / 0.1, c / 0.1):
        assert abs(np.mean(np.abs(xi) ** 2) - 1.0) < 0.05
        assert abs(np.mean(xi.real ** 2) - 0.5) < 0.05 and abs(np.mean(xi.imag ** 2) - 0.5) < 0.05
        assert abs(np.mean(xi)) < 0.03
    psi = inputs.gaussian_spinor(inputs.Grid(64, 64, 4.0, 4.0))
    assert np.allclose(m.add_noise(psi, 0.1, seed=7) - psi, a, atol=1e-15)
