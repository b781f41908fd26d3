"""Pins of the FP64 Fourier-neural-operator oracle (no GPU).

The spectral layer against numpy's FFT and against the identity on the kept
modes; every gradient against central finite differences of the loss; one
Adam step by hand; bfloat16 rounding on known values.
"""
import math

import numpy as np
import pytest

from oracle import fno


def rand_params(sh, seed=0, scale=0.4):
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, sh.size())


def test_spectral_layer_matches_numpy_fft():
    n, M, W = 16, 3, 2
    rng = np.random.default_rng(1)
    v = rng.standard_normal((2, W, n, n))
    R = rng.standard_normal((2 * M, M, W, W, 2))
    s, vh = fno.spectral(v, R, n, M)
    ky = fno.kept_ky(n, M)
    F = np.fft.fft2(v)                                   # [b][c][ky][kx]
    assert np.allclose(vh, F[:, :, ky][:, :, :, :M], atol=1e-10)
    Rc = R[..., 0] + 1j * R[..., 1]
    Z = np.zeros((2, W, n, n), complex)
    for j, k in enumerate(ky):
        for kx in range(M):
            Z[:, :, k, kx] = np.einsum("oc,bc->bo", Rc[j, kx], F[:, :, k, kx]) * (1.0 if kx == 0 else 2.0)
    assert np.allclose(s, np.fft.ifft2(Z).real, atol=1e-12)


def test_spectral_layer_is_the_identity_on_kept_modes():
    n, M, W = 16, 4, 1
    R = np.zeros((2 * M, M, W, W, 2))
    R[..., 0, 0, 0] = 1.0
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for kx, ky in [(0, 0), (1, 0), (0, 2), (3, 1), (2, -3), (3, -4)]:
        v = np.cos(2 * np.pi * (kx * x + ky * y) / n + 0.3)[None, None]
        s, _ = fno.spectral(v, R, n, M)
        assert np.allclose(s, v, atol=1e-12), (kx, ky)
    v = np.cos(2 * np.pi * (5 * x + 1 * y) / n)[None, None]  # kx = 5 not kept
    assert np.abs(fno.spectral(v, R, n, M)[0]).max() < 1e-12


def test_gelu_values():
    assert fno.gelu(np.array(0.0)) == 0.0
    assert abs(fno.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    x = np.linspace(-3, 3, 13)
    num = (fno.gelu(x + 1e-6) - fno.gelu(x - 1e-6)) / 2e-6
    assert np.allclose(fno.gelu_grad(x), num, atol=1e-8)


@pytest.mark.parametrize("L", [1, 2])
def test_gradients_match_finite_differences(L):
    sh = fno.Shapes(cin=2, cout=2, width=3, modes=2, layers=L, hidden=4)
    n, B = 8, 2
    rng = np.random.default_rng(7)
    a = rng.standard_normal((B, 2, n, n))
    target = rng.standard_normal((B, 2, n, n))
    th = rand_params(sh, 3)
    _, g = fno.loss_and_grad(sh, th, a, target)
    h = 1e-6
    idx = rng.choice(sh.size(), 60, replace=False)
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        num = (fno.loss(fno.forward(sh, th + e, a), target) - fno.loss(fno.forward(sh, th - e, a), target)) / (2 * h)
        assert abs(num - g[i]) < 1e-7 * max(1.0, abs(num)), (i, num, g[i])


def test_adam_first_step_by_hand():
    th, g = np.array([1.0, -2.0, 0.5]), np.array([0.3, -1e-3, 0.0])
    new, m, v = fno.adam_step(th, g, np.zeros(3), np.zeros(3), 1, 0.01)
    # t = 1: m_hat = g, v_hat = g^2, step = lr g / (|g| + eps)
    want = th - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(new, want, rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding():
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -3.14159265, 1e-30, 65504.0])
    want = np.array([1.0, 1.0, 1 + 2 ** -7, -3.140625, None, 65536.0], dtype=object)
    got = fno.round_bf16(vals)
    for gv, w, x in zip(got, want, vals):
        if w is None:
            assert abs(gv - x) <= 2 ** -8 * abs(x)
        else:
            assert gv == w, (x, gv, w)
