"""FP64 CPU oracle for the two-component TSSP step of arXiv:2010.15069.

TEST INFRASTRUCTURE ONLY: the slow, plain reference the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It shares no code with the CUDA path.

The arithmetic lives in ``spgpe_oracle.cpp`` (plain C++17, FP64, single thread,
its own radix-2 FFT); this module compiles it with the host compiler and wraps
it with ``ctypes``.  Every function takes and returns numpy arrays:
a spinor is a complex128 array of shape ``(2, ny, nx)`` (component up first,
x fastest), potentials are float64 ``(ny, nx)`` arrays or ``None`` for zero.

Model, grid and operator conventions are stated at the top of the C++ file
(Eq. 3 signs, Sec. 3.2 grid and splitting, Eq. 13 evolution operators).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgpe_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libspgpe_oracle.so")
_lock = threading.Lock()
_lib = None

NORM_TOTAL = 0
NORM_PER_COMPONENT = 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++ -O2, no fast-math); return its path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("xmax", ctypes.c_double), ("ymax", ctypes.c_double),
        ("V", ctypes.c_void_p), ("delta", ctypes.c_void_p), ("Omega", ctypes.c_void_p),
        ("g11", ctypes.c_double), ("g22", ctypes.c_double), ("g12", ctypes.c_double),
        ("kL", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_fft2.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
            lib.orc_apply.argtypes = [ctypes.POINTER(_Model), P, ctypes.c_double, ctypes.c_int, ctypes.c_int]
            lib.orc_step.argtypes = [ctypes.POINTER(_Model), P, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, P, P]
            lib.orc_norm.argtypes = [ctypes.POINTER(_Model), P, P]
            lib.orc_energy.argtypes = [ctypes.POINTER(_Model), P, P]
            lib.orc_observables.argtypes = [ctypes.POINTER(_Model), P, ctypes.c_int, P]
            lib.orc_add_noise.argtypes = [ctypes.POINTER(_Model), P, ctypes.c_double, ctypes.c_ulonglong,
                                          ctypes.c_long]
            for f in (lib.orc_fft2, lib.orc_apply, lib.orc_step, lib.orc_norm, lib.orc_energy,
                      lib.orc_observables, lib.orc_add_noise):
                f.restype = None
            lib.orc_splitmix64.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong]
            lib.orc_splitmix64.restype = ctypes.c_ulonglong
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Model:
    """Parameters of Eqs. 3-8 on an nx x ny grid over [-xmax, xmax) x [-ymax, ymax)."""

    def __init__(self, nx, ny, xmax, ymax, V=None, delta=None, Omega=None,
                 g11=0.0, g22=0.0, g12=0.0, kL=0.0):
        self.nx, self.ny, self.xmax, self.ymax = int(nx), int(ny), float(xmax), float(ymax)

        def arr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (self.ny, self.nx)))
            return a.copy()
        self.V, self.delta, self.Omega = arr(V), arr(delta), arr(Omega)
        self.g11, self.g22, self.g12, self.kL = float(g11), float(g22), float(g12), float(kL)
        self._c = _Model(self.nx, self.ny, self.xmax, self.ymax,
                         _ptr(self.V), _ptr(self.delta), _ptr(self.Omega),
                         self.g11, self.g22, self.g12, self.kL)

    @property
    def dx(self):
        return 2.0 * self.xmax / self.nx

    @property
    def dy(self):
        return 2.0 * self.ymax / self.ny

    def _psi(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        if psi.shape != (2, self.ny, self.nx):
            raise ValueError(f"spinor shape {psi.shape} != (2, {self.ny}, {self.nx})")
        return psi.copy()

    def step(self, psi, dt, nsteps, imag=False, norm_mode=NORM_TOTAL, target=(0.5, 0.5),
             residual=False):
        """Return the spinor after ``nsteps`` Strang steps (and the last-step residual)."""
        out = self._psi(psi)
        tgt = np.asarray(target, dtype=np.float64)
        res = np.zeros(1)
        _load().orc_step(ctypes.byref(self._c), _ptr(out), float(dt), int(nsteps), int(bool(imag)),
                         int(norm_mode), _ptr(tgt), _ptr(res) if residual else None)
        return (out, float(res[0])) if residual else out

    def apply(self, psi, tau, which, imag=False):
        """Apply one sub-operator: 'D', 'X', 'R' or 'K' (K includes F and F^-1)."""
        code = {"D": 0, "X": 1, "R": 2, "K": 3}[which]
        out = self._psi(psi)
        _load().orc_apply(ctypes.byref(self._c), _ptr(out), float(tau), int(bool(imag)), code)
        return out

    def norm(self, psi):
        psi = self._psi(psi)
        out = np.zeros(2)
        _load().orc_norm(ctypes.byref(self._c), _ptr(psi), _ptr(out))
        return out

    def energy(self, psi):
        psi = self._psi(psi)
        out = np.zeros(6)
        _load().orc_energy(ctypes.byref(self._c), _ptr(psi), _ptr(out))
        return out


    def observables(self, psi, npts=None):
        """{s (Eq. 14), n_up, n_dn (Eq. 15 windings), R99} as a length-4 array; the
        contour has 4 max(nx, ny) points unless npts is given."""
        psi = self._psi(psi)
        out = np.zeros(4)
        _load().orc_observables(ctypes.byref(self._c), _ptr(psi), int(npts or 4 * max(self.nx, self.ny)), _ptr(out))
        return out

    def add_noise(self, psi, sigma, seed, inst=0):
        """psi + sigma xi, xi complex standard normal from the counter-based SplitMix64 stream."""
        out = self._psi(psi)
        _load().orc_add_noise(ctypes.byref(self._c), _ptr(out), float(sigma), int(seed) & (2 ** 64 - 1), int(inst))
        return out


def splitmix64(seed, c):
    """Draw c of the oracle's counter-based SplitMix64 stream `seed`."""
    return int(_load().orc_splitmix64(int(seed) & (2 ** 64 - 1), int(c)))


def fft2(plane, inverse=False):
    """The oracle's own 2D FFT of one complex (ny, nx) plane, unnormalised."""
    a = np.ascontiguousarray(plane, dtype=np.complex128).copy()
    ny, nx = a.shape
    _load().orc_fft2(nx, ny, _ptr(a), +1 if inverse else -1)
    return a
