"""The single-precision elementary functions of the pointwise operators
(``csrc/fastmath.cuh``: Taylor series with Cody-Waite range reduction) against
FP64 references, over every tier and the tier boundaries.

The parity cases keep the substep phases small, so the range-reduced tiers
are reached there only by a few points; this sweep evaluates each function on
the GPU (a probe kernel built from the library's own header) at dense
arguments up to the documented range and compares it with numpy's FP64
functions of the same float arguments.  Bounds (the header's): exp(2ih) - 1
within 2.5e-7 relative to |w|; expm1 within 1.5e-7 relative (expm1_small,
below |x| = 1/2: 1e-7; expm1_quarter, below |x| = 1/4: 1.5e-7); the shear
constants rotate a unit vector by 2h within 3e-7.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc", "fastmath_probe.cu")
CSRC = os.path.join(ROOT, "paper_2010_15069_gb300", "csrc")
LIB = os.path.join(HERE, "_build", "libfastmath_probe.so")
PIO2 = np.pi / 2


@pytest.fixture(scope="module")
def probe():
    from paper_2010_15069_gb300 import build
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    deps = [SRC, os.path.join(CSRC, "fastmath.cuh")]
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(d) for d in deps):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([build.nvcc(), "-std=c++17", "-O3", *build.ARCH, "-Xcompiler", "-fPIC", "-shared",
                        "-I", CSRC, SRC, "-o", tmp], check=True)
        os.replace(tmp, LIB)
    lib = ctypes.CDLL(LIB)
    lib.fastmath_probe.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.fastmath_probe.restype = ctypes.c_int

    def run(fn, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        xd = torch.from_numpy(x).cuda()
        out = torch.zeros(3 * x.size, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        assert lib.fastmath_probe(fn, xd.data_ptr(), x.size, out.data_ptr()) == 0
        return x.astype(np.float64), out.cpu().numpy().astype(np.float64).reshape(-1, 3)
    return run


def around(points, n=64):
    """Floats just below and above each point (n ulps either way), both signs."""
    out = []
    for p in points:
        v = np.float32(p)
        lo, hi = v, v
        for _ in range(n):
            lo, hi = np.nextafter(lo, np.float32(-np.inf)), np.nextafter(hi, np.float32(np.inf))
            out += [lo, hi]
        out.append(v)
    out = np.array(out, dtype=np.float32)
    return np.concatenate([out, -out])


def logspace_both(lo, hi, n):
    a = np.logspace(lo, hi, n)
    return np.concatenate([a, -a])


def rotation_error(t, s, neg, h):
    """Largest error of the three-shear rotation (t, s, negation) applied in FP64
    to the unit vectors, against the exact rotation by 2h."""
    c2, s2 = np.cos(2.0 * h), np.sin(2.0 * h)
    sg = np.where(neg > 0.5, -1.0, 1.0)
    # (1, 0) -> (1 - t s, s); (0, 1) -> (-2t + s t^2, 1 - s t)
    e1 = np.hypot(sg * (1.0 - t * s) - c2, sg * s - s2)
    e2 = np.hypot(sg * (-2.0 * t + s * t * t) + s2, sg * (1.0 - s * t) - c2)
    return np.maximum(e1, e2)


def test_expi2_m1_all_tiers(probe):
    """w = exp(2ih) - 1: the direct series below |h| = 1/8, the reduced one above,
    up to |h| = 3000, near the tier boundary and near multiples of pi/2."""
    x = np.concatenate([np.linspace(-3000.0, 3000.0, 600001), logspace_both(-30, -0.9, 4001),
                        around([0.125]),
                        ((PIO2 * np.arange(-1900, 1901))[:, None] + np.linspace(-1e-3, 1e-3, 5)[None, :]).ravel(),
                        (PIO2 * np.arange(-1900, 1901)).astype(np.float32)])
    h, out = probe(0, x)
    w = (-2.0 * np.sin(h) ** 2) + 1j * np.sin(2.0 * h)
    err = np.abs(out[:, 0] + 1j * out[:, 1] - w)
    bound = 2.5e-7 * np.abs(w) + 4e-13
    worst = np.argmax(err / bound)
    assert np.all(err <= bound), (h[worst], err[worst], np.abs(w[worst]))


def test_expm1_f_all_tiers(probe):
    """expm1: the series below |x| = 1/16 and the reduced form from -87 to 88;
    saturation to -1 below and a finite value above."""
    x = np.concatenate([np.linspace(-87.0, 88.0, 400001), logspace_both(-30, -1, 4001), around([0.0625, 0.5])])
    xd, out = probe(1, x)
    ref = np.expm1(xd)
    err = np.abs(out[:, 0] - ref)
    worst = np.argmax(err / np.abs(ref))
    assert np.all(err <= 1.5e-7 * np.abs(ref)), (xd[worst], err[worst] / abs(ref[worst]))
    _, sat = probe(1, np.array([-100.0, -88.5, 100.0, 1e30], dtype=np.float32))
    assert np.all(np.abs(sat[:2, 0] + 1.0) <= 1e-7)
    assert np.all(np.isfinite(sat[2:, 0])) and np.all(sat[2:, 0] > 1e38)


def test_expm1_small(probe):
    """expm1 for |x| < 1/2 (the imaginary-time D factors of warps whose phases
    are all below the bound)."""
    x = np.concatenate([np.linspace(-0.5, 0.5, 200001)[1:-1], logspace_both(-30, np.log10(0.49), 4001)])
    xd, out = probe(2, x)
    ref = np.expm1(xd)
    err = np.abs(out[:, 0] - ref)
    assert np.all(err <= 1e-7 * np.abs(ref)), xd[np.argmax(err / np.abs(ref))]


def test_expm1_quarter(probe):
    """expm1 for |x| < 1/4 (the imaginary-time D factors of warps whose
    interaction exponents are all below the bound): the series to x^6/6!,
    truncation below 4.8e-8 relative."""
    x = np.concatenate([np.linspace(-0.25, 0.25, 200001)[1:-1], logspace_both(-30, np.log10(0.249), 4001)])
    xd, out = probe(6, x)
    ref = np.expm1(xd)
    err = np.abs(out[:, 0] - ref)
    assert np.all(err <= 1.5e-7 * np.abs(ref)), xd[np.argmax(err / np.abs(ref))]


def test_shear_constants_general_all_tiers(probe):
    """t = tan r, s = sin 2r with r the reduced half phase and a negation for odd
    multiples of pi/2: the cubic series below |h| = 1/32, the quintic one below
    1/8, the reduced form above, up to |h| < 2^12 pi/2 (the range of an exact
    reduction)."""
    top = 4096 * PIO2 * 0.999
    x = np.concatenate([np.linspace(-top, top, 800001), logspace_both(-30, -0.5, 4001),
                        around([1.0 / 32.0, 0.125, np.pi / 4, 3 * np.pi / 4]),
                        (PIO2 * np.arange(-4000, 4001)).astype(np.float32)])
    h, out = probe(3, x)
    t, s, neg = out[:, 0], out[:, 1], out[:, 2]
    err = rotation_error(t, s, neg, h)
    worst = np.argmax(err)
    assert err.max() <= 3e-7, (h[worst], err[worst])
    # the reduced tier folds the rotation into |r| <= pi/4 (tan r within [-1, 1], up to the
    # rounding of h 2/pi to the nearest integer)
    big = np.abs(h) >= 0.125
    assert np.all(np.abs(t[big]) <= 1.01)
    # small half phases: relative accuracy of t and s themselves
    sm = (np.abs(h) < 0.125) & (h != 0)
    assert np.all(np.abs(t[sm] - np.tan(h[sm])) <= 2e-7 * np.abs(np.tan(h[sm])))
    assert np.all(np.abs(s[sm] - np.sin(2 * h[sm])) <= 2e-7 * np.abs(np.sin(2 * h[sm])))
    assert np.all(neg[sm] == 0)


@pytest.mark.parametrize("fn,limit", [(4, 0.125), (5, 1.0 / 64.0)])
def test_shear_constants_warp_uniform_tiers(probe, fn, limit):
    """The series a warp takes when every phase it holds is below the tier's
    bound (1/8: quintic-and-up series; 1/64: cubic series)."""
    x = np.concatenate([np.linspace(-limit, limit, 100001)[1:-1], logspace_both(-30, np.log10(limit) - 1e-3, 4001)])
    h, out = probe(fn, x)
    t, s = out[:, 0], out[:, 1]
    nz = h != 0
    assert np.all(np.abs(t[nz] - np.tan(h[nz])) <= 2e-7 * np.abs(np.tan(h[nz])))
    assert np.all(np.abs(s[nz] - np.sin(2 * h[nz])) <= 2e-7 * np.abs(np.sin(2 * h[nz])))
    assert rotation_error(t, s, np.zeros_like(t), h).max() <= 3e-7
