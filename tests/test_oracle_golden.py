"""The oracle and the Eq. 12 generator against values the paper prints
(tests/golden/gauge_potential_sec6.txt, Sec. 6; no GPU).

With spin-orbit coupling kL and a uniform Raman coupling Omega (delta = 0, no
interactions), the imaginary-time ground state in a weak trap along x sits in
the two minima of the lower dressed band: the k-space density of the oracle's
ground state peaks at kx = +-A*, the printed gauge-potential magnitude.  A
factor slip in the Raman term (Omega for Omega/2), in the kinetic SOC term or
in E_L moves those peaks by a large fraction of kL.  The Eq. 12 profile of the
spin-Hall generator makes A*(y) fall linearly from kL at y = 0 to 0 at y = 4,
as the paper states.
"""
import math
import os

import numpy as np
import pytest

from paper_2010_15069_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gauge_potential_sec6.txt")


def tables():
    out, cur = {}, None
    with open(GOLDEN) as fh:
        for ln in fh:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            if ln.startswith("["):
                cur = ln.strip("[]")
                out[cur] = []
            else:
                out[cur].append(tuple(float(v) for v in ln.split()))
    return out


def kspace_peak(psi, g, sign):
    """Position of the largest peak of the total k-space density along kx on
    the given side (quadratic interpolation around the largest bin)."""
    dens = (np.abs(np.fft.fft(psi[0], axis=1)) ** 2 + np.abs(np.fft.fft(psi[1], axis=1)) ** 2).sum(axis=0)
    n = g.nx
    f = np.arange(n)
    k = 2 * np.pi * np.where(f < n // 2, f, f - n) / (2 * g.xmax)
    side = k * sign > 0
    i = int(np.argmax(np.where(side, dens, -1.0)))
    y0, y1, y2 = dens[i - 1], dens[i], dens[(i + 1) % n]
    return k[i] + 0.5 * (k[1] - k[0]) * (y0 - y2) / (y0 - 2 * y1 + y2)


def test_golden_table_follows_the_printed_formula():
    t = tables()
    for ratio, a in t["minima"]:
        assert abs(a - math.sqrt(1.0 - ratio * ratio)) < 1e-15
    ys = [y for y, _ in t["eq12"]]
    assert ys[0] == 0.0 and ys[-1] == 4.0


@pytest.mark.parametrize("row", range(3))
def test_dressed_band_minima_at_the_printed_gauge_potential(orc, row):
    ratio, a_over_kl = tables()["minima"][row]
    kL = 2.0
    E_L = kL * kL / 2
    Om = ratio * 4.0 * E_L
    g = inputs.Grid(512, 8, 40.0, 1.0)
    X, _ = g.mesh()
    V = 0.5 * 0.1 ** 2 * X * X           # weak trap along x only: the minima stay resolved in k
    m = orc.Model(g.nx, g.ny, g.xmax, g.ymax, V=V, Omega=np.full((g.ny, g.nx), Om), kL=kL)
    psi = m.step(inputs.gaussian_spinor(g, width=5.0, noise=1e-3, seed=3), 0.05, 2000, imag=True,
                 norm_mode=0, target=(0.5, 0.5))
    astar = a_over_kl * kL
    for sign in (1, -1):
        assert abs(sign * kspace_peak(psi, g, sign) - astar) < 0.02 * kL, (ratio, sign)
    # Eq. 3's sign: the up component lives at kx > 0 (the dressed minimum at +A*)
    up_k = np.abs(np.fft.fft(psi[0], axis=1)) ** 2
    f = np.arange(g.nx)
    kpos = np.where(f < g.nx // 2, f, f - g.nx) > 0
    assert up_k[:, kpos].sum() > up_k[:, ~kpos].sum()


def test_eq12_profile_makes_the_gauge_potential_linear():
    t = tables()["eq12"]
    E_L = 2.0
    g = inputs.Grid(8, 64, 4.0, 8.0)         # y from -8 to 8 in steps of 0.25
    om = inputs.raman_profile_y(g, E_L)
    for y, a_over_kl in t:
        j = int(np.argmin(np.abs(g.y - y)))
        assert abs(g.y[j] - y) < 1e-12
        ratio = om[j] / (4.0 * E_L)
        assert abs(math.sqrt(max(0.0, 1.0 - ratio * ratio)) - a_over_kl) < 1e-12, y
