"""Data preparation of the learned warm start (host side, numpy).

The FNO (``paper_2010_15069_gb300.FNO``) maps input fields built from the
parameters of a sweep instance to the instance's ground state; this module
builds those fields and brings ground states to and from the network's
output channels.  Nothing here computes any part of the time-splitting
method: the ground states come from the library's relaxation, the network
runs in the library's kernels.

Input channels (CIN = 6), on the instance's grid over [-xmax, xmax) x
[-ymax, ymax): x / xmax, y / ymax, the detuning delta' y / ymax, Omega / 6,
(ln g - ln 50) / (ln 2000 - ln 50), 5 (g12 / g - 1), the last three constant.
Output channels (COUT = 4): SCALE x (Re psi_up, Im psi_up, Re psi_dn,
Im psi_dn) of the ground state with its global phase fixed so that
sum (psi_up + psi_dn) is real and positive.
"""
from __future__ import annotations

import math

import numpy as np

CIN, COUT, SCALE = 6, 4, 10.0


def features(grid, g, g12, Omega, delta_slope):
    X, Y = grid.mesh()
    one = np.ones_like(X)
    return np.stack([X / grid.xmax, Y / grid.ymax, delta_slope * Y / grid.ymax, (Omega / 6.0) * one,
                     ((math.log(g) - math.log(50.0)) / (math.log(2000.0) - math.log(50.0))) * one,
                     5.0 * (g12 / g - 1.0) * one]).astype(np.float32)


def gauge_fix(psi):
    """psi [2][ny][nx] times the global phase that makes sum(psi_up + psi_dn) real and positive."""
    z = psi[0].sum() + psi[1].sum()
    return psi * (np.conj(z) / abs(z)) if abs(z) > 0 else psi


def to_channels(psi):
    psi = gauge_fix(psi)
    return (SCALE * np.stack([psi[0].real, psi[0].imag, psi[1].real, psi[1].imag])).astype(np.float32)


def from_channels(ch):
    ch = np.asarray(ch, dtype=np.float64) / SCALE
    return np.stack([ch[0] + 1j * ch[1], ch[2] + 1j * ch[3]])
