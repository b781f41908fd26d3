"""FP64 reference of the Fourier neural operator used as the ground-state warm start.

TEST INFRASTRUCTURE ONLY: the plain numpy definition the CUDA training and
inference kernels are checked against (forward, loss, every gradient, one Adam
step).  Only ``tests/`` and the benchmark's CPU leg may import it; it shares
no code with the CUDA path.

The network (the Fourier neural operator of Li et al., arXiv:2010.08895, with
the sizes of the learned warm start: width W = 64, M = 32 modes, 4 Fourier
layers; the paper itself has no learned part) maps input fields
a[c_in][n][n] to output fields out[c_out][n][n]:

    v_0 = P a + p                                   (pointwise, W x c_in)
    u_l = W_l v_l + w_l + S_l(v_l),  v_{l+1} = gelu(u_l)  (l < L-1),  v_L = u_{L-1}
    out = Q2 gelu(Q1 v_L + q1) + q2                 (pointwise, hidden H)

with the exact GELU x Phi(x) and the spectral convolution

    vh[c][j][kx] = sum_{y,x} v[c][y][x] exp(-2 pi i (kx x + ky_j y) / n)
    oh[o][j][kx] = sum_c R[j][kx][o][c] vh[c][j][kx]
    S(v)[o][y][x] = Re sum_{j,kx} g_kx oh[o][j][kx] exp(+2 pi i (kx x + ky_j y) / n) / n^2

over the kept modes kx = 0..M-1 and ky_j = j (j < M) or n - 2M + j (j >= M),
with g_0 = 1 and g_kx = 2 otherwise (the real field of a half spectrum).  The
loss of a batch is the mean relative squared error
sum_b ||out_b - target_b||^2 / ||target_b||^2 / B.

Parameters are one flat vector, in this order: P [W][c_in], p [W]; per layer
W_l [W][W], w_l [W], R_l [2M][M][W][W][2] (real, imaginary); Q1 [H][W],
q1 [H], Q2 [c_out][H], q2 [c_out].
"""
from __future__ import annotations

import math

import numpy as np

try:
    from scipy.special import erf as _erf
except ImportError:  # pragma: no cover
    _erf = np.vectorize(math.erf)


class Shapes:
    def __init__(self, cin, cout, width, modes, layers, hidden):
        self.cin, self.cout, self.W, self.M, self.L, self.H = cin, cout, width, modes, layers, hidden

    def layout(self):
        """[(name, shape)] of the flat parameter vector."""
        W, M, H = self.W, self.M, self.H
        out = [("P", (W, self.cin)), ("p", (W,))]
        for l in range(self.L):
            out += [(f"W{l}", (W, W)), (f"w{l}", (W,)), (f"R{l}", (2 * M, M, W, W, 2))]
        out += [("Q1", (H, W)), ("q1", (H,)), ("Q2", (self.cout, H)), ("q2", (self.cout,))]
        return out

    def size(self):
        return sum(int(np.prod(s)) for _, s in self.layout())

    def unpack(self, flat):
        d, o = {}, 0
        for name, shape in self.layout():
            k = int(np.prod(shape))
            d[name] = np.asarray(flat[o:o + k], dtype=np.float64).reshape(shape)
            o += k
        return d

    def pack(self, d):
        return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in self.layout()])


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def kept_ky(n, M):
    return np.concatenate([np.arange(M), np.arange(n - M, n)])


def dft_mats(n, M):
    """Ex[x, kx] = exp(-2 pi i kx x / n) (kx < M); Ey[j, y] = exp(-2 pi i ky_j y / n)."""
    x = np.arange(n)
    Ex = np.exp(-2j * np.pi * np.outer(x, np.arange(M)) / n)
    Ey = np.exp(-2j * np.pi * np.outer(kept_ky(n, M), x) / n)
    g = np.where(np.arange(M) == 0, 1.0, 2.0)
    return Ex, Ey, g


def spectral(v, R, n, M):
    """S(v) for v [B][W][n][n]; also returns vh (for the backward pass)."""
    Ex, Ey, g = dft_mats(n, M)
    vh = np.einsum("jy,bcyx,xk->bcjk", Ey, v, Ex, optimize=True)
    Rc = R[..., 0] + 1j * R[..., 1]                            # [2M][M][o][c]
    oh = np.einsum("jkoc,bcjk->bojk", Rc, vh, optimize=True)
    s = np.einsum("jy,bojk,xk->boyx", np.conj(Ey), oh * g, np.conj(Ex), optimize=True).real / (n * n)
    return s, vh


def spectral_back(ds, vh, R, n, M):
    """Gradients of S: (dv, dR) for ds [B][W][n][n]."""
    Ex, Ey, g = dft_mats(n, M)
    doh = np.einsum("jy,boyx,xk->bojk", Ey, ds, Ex, optimize=True) * g / (n * n)   # dL/dRe + i dL/dIm of oh
    Rc = R[..., 0] + 1j * R[..., 1]
    dRc = np.einsum("bojk,bcjk->jkoc", doh, np.conj(vh), optimize=True)
    dvh = np.einsum("jkoc,bojk->bcjk", np.conj(Rc), doh, optimize=True)
    dv = np.einsum("jy,bcjk,xk->bcyx", np.conj(Ey), dvh, np.conj(Ex), optimize=True).real
    return dv, np.stack([dRc.real, dRc.imag], axis=-1)


def pointwise(Wm, b, v):
    return np.einsum("oc,bcyx->boyx", Wm, v, optimize=True) + b[None, :, None, None]


def forward(sh, flat, a, keep=False):
    """out [B][c_out][n][n] for a [B][c_in][n][n] (and the saved activations)."""
    P = sh.unpack(flat)
    n, M = a.shape[-1], sh.M
    v = pointwise(P["P"], P["p"], a)
    vs, us, vhs = [v], [], []
    for l in range(sh.L):
        s, vh = spectral(v, P[f"R{l}"], n, M)
        u = pointwise(P[f"W{l}"], P[f"w{l}"], v) + s
        us.append(u)
        vhs.append(vh)
        v = gelu(u) if l < sh.L - 1 else u
        vs.append(v)
    hp = pointwise(P["Q1"], P["q1"], v)
    h = gelu(hp)
    out = pointwise(P["Q2"], P["q2"], h)
    return (out, dict(vs=vs, us=us, vhs=vhs, hp=hp, h=h)) if keep else out


def loss(out, target):
    B = out.shape[0]
    num = ((out - target) ** 2).reshape(B, -1).sum(1)
    den = (target ** 2).reshape(B, -1).sum(1)
    return float((num / den).mean())


def loss_and_grad(sh, flat, a, target):
    """(loss, flat gradient) of the mean relative squared error."""
    P = sh.unpack(flat)
    B, n, M = a.shape[0], a.shape[-1], sh.M
    out, st = forward(sh, flat, a, keep=True)
    den = (target ** 2).reshape(B, -1).sum(1)
    dout = 2.0 * (out - target) / den[:, None, None, None] / B
    G = {}
    G["Q2"] = np.einsum("boyx,bhyx->oh", dout, st["h"], optimize=True)
    G["q2"] = dout.sum(axis=(0, 2, 3))
    dh = np.einsum("oh,boyx->bhyx", P["Q2"], dout, optimize=True)
    dhp = dh * gelu_grad(st["hp"])
    v = st["vs"][-1]
    G["Q1"] = np.einsum("bhyx,bcyx->hc", dhp, v, optimize=True)
    G["q1"] = dhp.sum(axis=(0, 2, 3))
    dv = np.einsum("hc,bhyx->bcyx", P["Q1"], dhp, optimize=True)
    for l in reversed(range(sh.L)):
        du = dv * gelu_grad(st["us"][l]) if l < sh.L - 1 else dv
        vl = st["vs"][l]
        G[f"W{l}"] = np.einsum("boyx,bcyx->oc", du, vl, optimize=True)
        G[f"w{l}"] = du.sum(axis=(0, 2, 3))
        dvs, dR = spectral_back(du, st["vhs"][l], P[f"R{l}"], n, M)
        G[f"R{l}"] = dR
        dv = np.einsum("oc,boyx->bcyx", P[f"W{l}"], du, optimize=True) + dvs
    G["P"] = np.einsum("boyx,bcyx->oc", dv, a, optimize=True)
    G["p"] = dv.sum(axis=(0, 2, 3))
    return loss(out, target), sh.pack(G)


def adam_step(flat, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, 2015) with bias correction; t counts from 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)
