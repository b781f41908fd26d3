"""GB300 (sm_103a) solver for the two-component quasi-2D GPE of arXiv:2010.15069.

The hot path is the Strang time-splitting spectral step (Sec. 3.2, Eq. 13)
run by hand-written CUDA kernels in ``libspgpe.so`` behind the C ABI of
``include/spgpe.h``.  This package is the thin Python binding:

* ``spgpe_*`` functions with the C names, taking raw pointers (``int``),
  raising :class:`SpgpeError` on a negative status;
* :class:`Context`, which takes torch CUDA tensors (device spinors, stepped
  in place on the context's stream) or numpy arrays (host spinors, staged by
  the library) and returns numpy results.

PyTorch is used only for device memory and streams.  Nothing here computes
any part of the method; importing works without the library, but every call
needs it built (``paper_2010_15069_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import (SPGPE_C64, SPGPE_C128, SPGPE_NORM_PER_COMPONENT, SPGPE_NORM_TOTAL, SPGPE_RELAX_GIVE_UP, SPGPE_RELAX_LAGGED, SPGPE_IMAG_LAGGED,
                   SPGPE_RELAX_LADDER, SpgpeError, check, load, SPGPE_OK, SPGPE_ETIMEOUT)

__all__ = [
    "SPGPE_C64", "SPGPE_C128", "SPGPE_OK", "SPGPE_ETIMEOUT", "SPGPE_NORM_TOTAL", "SPGPE_NORM_PER_COMPONENT", "SPGPE_RELAX_LADDER", "SPGPE_RELAX_GIVE_UP",
    "SPGPE_RELAX_LAGGED", "SPGPE_IMAG_LAGGED",
    "SpgpeError",
    "Context", "FNO", "load",
    "spgpe_init_grid", "spgpe_init_batch", "spgpe_init_multi", "spgpe_set_potentials", "spgpe_set_potentials_separable",
    "spgpe_step_real", "spgpe_step_imag", "spgpe_relax", "spgpe_autotune", "spgpe_observables", "spgpe_add_noise", "spgpe_energy", "spgpe_norm", "spgpe_sync", "spgpe_wait_probe",
    "spgpe_cufft_step_real", "spgpe_probe_ceilings", "spgpe_destroy", "spgpe_last_error", "spgpe_version",
    "spgpe_last_launches", "spgpe_set_timing", "spgpe_timing",
]


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------ C-name layer

def spgpe_init_grid(nx, ny, xmax, ymax, dtype=SPGPE_C64, stream=0):
    ctx = ctypes.c_void_p()
    check(load().spgpe_init_grid(ctypes.byref(ctx), int(nx), int(ny), float(xmax), float(ymax),
                                 int(dtype), ctypes.c_void_p(int(stream))))
    return ctx.value


def spgpe_init_batch(nx, ny, xmax, ymax, ninst, dtype=SPGPE_C64, stream=0):
    ctx = ctypes.c_void_p()
    check(load().spgpe_init_batch(ctypes.byref(ctx), int(nx), int(ny), float(xmax), float(ymax),
                                  int(ninst), int(dtype), ctypes.c_void_p(int(stream))))
    return ctx.value


def spgpe_init_multi(classes, dtype=SPGPE_C64, stream=0):
    """classes: sequence of (nx, ny, ninst, xmax, ymax), one per grid size."""
    k = len(classes)
    nx = np.array([c[0] for c in classes], dtype=np.int32)
    ny = np.array([c[1] for c in classes], dtype=np.int32)
    ni = np.array([c[2] for c in classes], dtype=np.int32)
    xm = np.array([c[3] for c in classes], dtype=np.float64)
    ym = np.array([c[4] for c in classes], dtype=np.float64)
    ctx = ctypes.c_void_p()
    check(load().spgpe_init_multi(ctypes.byref(ctx), k, *(a.ctypes.data_as(ctypes.c_void_p) for a in (nx, ny, ni, xm, ym)),
                                  int(dtype), ctypes.c_void_p(int(stream))))
    return ctx.value


def spgpe_set_potentials(ctx, V=None, delta=None, Omega=None, g11=0.0, g22=0.0, g12=0.0, kL=0.0):
    V, delta, Omega = _f64(V), _f64(delta), _f64(Omega)
    check(load().spgpe_set_potentials(ctx, _ptr(V), _ptr(delta), _ptr(Omega), float(g11), float(g22),
                                      float(g12), float(kL)), ctx)


def spgpe_set_potentials_separable(ctx, inst, Vx=None, Vy=None, delta_x=None, delta_y=None, Omega_x=None,
                                   Omega_y=None, g11=0.0, g22=0.0, g12=0.0, kL=0.0):
    arrs = [_f64(a) for a in (Vx, Vy, delta_x, delta_y, Omega_x, Omega_y)]
    check(load().spgpe_set_potentials_separable(ctx, int(inst), *[_ptr(a) for a in arrs], float(g11),
                                                float(g22), float(g12), float(kL)), ctx)


def spgpe_step_real(ctx, psi_ptr, dt, nsteps):
    check(load().spgpe_step_real(ctx, ctypes.c_void_p(int(psi_ptr)), float(dt), int(nsteps)), ctx)


def spgpe_step_imag(ctx, psi_ptr, dtau, nsteps, norm_mode=SPGPE_NORM_TOTAL, target=(0.5, 0.5),
                    residual=False, ninst=1):
    tgt = _f64(target, 2)
    res = np.zeros(int(ninst)) if residual else None
    check(load().spgpe_step_imag(ctx, ctypes.c_void_p(int(psi_ptr)), float(dtau), int(nsteps), int(norm_mode),
                                 _ptr(tgt), _ptr(res)), ctx)
    return res


def spgpe_relax(ctx, psi_ptr, dtau, tol, max_steps, check_every=200, norm_mode=SPGPE_NORM_TOTAL,
                target=(0.5, 0.5), flags=0, handoff=0.0, ninst=1):
    """Returns (residuals per instance, (steps in complex64, steps in the context's precision))."""
    tgt = _f64(target, 2)
    res = np.zeros(int(ninst))
    steps = np.zeros(2, dtype=np.int32)
    check(load().spgpe_relax(ctx, ctypes.c_void_p(int(psi_ptr)), float(dtau), float(tol), int(max_steps),
                             int(check_every), int(norm_mode), _ptr(tgt), int(flags), float(handoff), _ptr(res),
                             steps.ctypes.data_as(ctypes.c_void_p)), ctx)
    return res, (int(steps[0]), int(steps[1]))


def spgpe_autotune(ctx, psi_ptr, dt, nclass=1):
    """Returns (chosen variant per class, ms per step per class)."""
    ch = np.zeros(int(nclass), dtype=np.int32)
    ms = np.zeros(int(nclass))
    check(load().spgpe_autotune(ctx, ctypes.c_void_p(int(psi_ptr)), float(dt), ch.ctypes.data_as(ctypes.c_void_p),
                                _ptr(ms)), ctx)
    return ch, ms


def spgpe_observables(ctx, psi_ptr, ninst=1):
    """(ninst, 4) array of {s (Eq. 14), n_up, n_dn (Eq. 15 windings), R99}."""
    out = np.zeros((int(ninst), 4))
    check(load().spgpe_observables(ctx, ctypes.c_void_p(int(psi_ptr)), _ptr(out)), ctx)
    return out


def spgpe_add_noise(ctx, psi_ptr, sigma, seed):
    check(load().spgpe_add_noise(ctx, ctypes.c_void_p(int(psi_ptr)), float(sigma),
                                 ctypes.c_ulonglong(int(seed) & (2 ** 64 - 1))), ctx)


def spgpe_energy(ctx, psi_ptr, ninst=1):
    out = np.zeros((int(ninst), 6))
    check(load().spgpe_energy(ctx, ctypes.c_void_p(int(psi_ptr)), _ptr(out)), ctx)
    return out


def spgpe_norm(ctx, psi_ptr, ninst=1):
    out = np.zeros((int(ninst), 2))
    check(load().spgpe_norm(ctx, ctypes.c_void_p(int(psi_ptr)), _ptr(out)), ctx)
    return out


def spgpe_sync(ctx):
    check(load().spgpe_sync(ctx), ctx)


def spgpe_wait_probe(ctx, cycles):
    """Run the bounded-wait failure probe; returns the status code (SPGPE_ETIMEOUT
    when the wait gave up and was reported, as it should)."""
    return int(load().spgpe_wait_probe(ctx, int(cycles)))


def spgpe_cufft_step_real(ctx, psi_ptr, dt, nsteps):
    check(load().spgpe_cufft_step_real(ctx, ctypes.c_void_p(int(psi_ptr)), float(dt), int(nsteps)), ctx)


def spgpe_probe_ceilings():
    """This GPU's measured ceilings (microbenchmarks; see include/spgpe.h)."""
    from ._lib import PROBE_SIZES_MIB
    out = np.zeros(4 + len(PROBE_SIZES_MIB))
    check(load().spgpe_probe_ceilings(_ptr(out), out.size))
    return {"fp32_fma_tflops": float(out[0]), "fp64_fma_tflops": float(out[1]),
            "sincosf_gcalls_per_s": float(out[2]), "copy_gbs": float(out[3]),
            "read_gbs_by_working_set_mib": {int(m): float(v) for m, v in zip(PROBE_SIZES_MIB, out[4:])}}


def spgpe_destroy(ctx):
    load().spgpe_destroy(ctx)


def spgpe_last_error(ctx=None):
    m = load().spgpe_last_error(ctx)
    return m.decode() if m else ""


def spgpe_version():
    return load().spgpe_version()


def spgpe_last_launches(ctx):
    return load().spgpe_last_launches(ctx)


def spgpe_set_timing(ctx, enable):
    check(load().spgpe_set_timing(ctx, int(bool(enable))), ctx)


def spgpe_timing(ctx):
    """{kind name: (launches, summed ms)} since timing was enabled (or last read)."""
    from ._lib import KIND_NAMES, NKINDS
    ms = np.zeros(NKINDS)
    cnt = np.zeros(NKINDS, dtype=np.int32)
    check(load().spgpe_timing(ctx, _ptr(ms), _ptr(cnt)), ctx)
    return {KIND_NAMES[k]: (int(cnt[k]), float(ms[k])) for k in range(NKINDS) if cnt[k]}


# ------------------------------------------------------------ learned warm start

class FNO:
    """The Fourier neural operator of the warm start (spgpe_fno_*): torch float32
    CUDA tensors in and out, laid out [batch][channel][n][n]; parameters as a
    numpy float32 vector in the layout documented in include/spgpe.h."""

    def __init__(self, cin, cout, width=64, modes=32, layers=4, hidden=128, seed=0, stream=None):
        self.cin, self.cout, self.width, self.modes, self.layers, self.hidden = cin, cout, width, modes, layers, hidden
        s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
        h = ctypes.c_void_p()
        rc = load().spgpe_fno_create(ctypes.byref(h), int(cin), int(cout), int(width), int(modes), int(layers),
                                     int(hidden), ctypes.c_ulonglong(int(seed) & (2 ** 64 - 1)), ctypes.c_void_p(s))
        if rc != 0:
            raise SpgpeError(rc, "spgpe_fno_create failed")
        self._h = h.value

    def _check(self, rc):
        if rc != 0:
            msg = load().spgpe_fno_last_error(self._h)
            raise SpgpeError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            load().spgpe_fno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def num_params(self):
        return int(load().spgpe_fno_num_params(self._h))

    def get_params(self):
        out = np.zeros(self.num_params(), dtype=np.float32)
        self._check(load().spgpe_fno_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        if theta.size != self.num_params():
            raise ValueError("parameter vector of the wrong length")
        self._check(load().spgpe_fno_set_params(self._h, theta.ctypes.data_as(ctypes.c_void_p)))

    @staticmethod
    def _dev(t, ch):
        import torch  # device memory only
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.dim() != 4 or t.shape[1] != ch \
                or t.shape[2] != t.shape[3]:
            raise ValueError(f"expected a contiguous CUDA float32 tensor [batch][{ch}][n][n]")
        return t.data_ptr()

    def forward(self, a):
        import torch
        out = torch.empty((a.shape[0], self.cout, a.shape[2], a.shape[3]), dtype=torch.float32, device=a.device)
        self._check(load().spgpe_fno_forward(self._h, ctypes.c_void_p(self._dev(a, self.cin)), int(a.shape[0]),
                                             int(a.shape[2]), ctypes.c_void_p(out.data_ptr())))
        return out

    def gradient(self, a, target):
        """(loss, gradient as a numpy float32 vector, output tensor)."""
        import torch
        out = torch.empty_like(target)
        g = np.zeros(self.num_params(), dtype=np.float32)
        loss = ctypes.c_double()
        self._check(load().spgpe_fno_gradient(self._h, ctypes.c_void_p(self._dev(a, self.cin)),
                                              ctypes.c_void_p(self._dev(target, self.cout)), int(a.shape[0]),
                                              int(a.shape[2]), ctypes.c_void_p(out.data_ptr()), ctypes.byref(loss),
                                              g.ctypes.data_as(ctypes.c_void_p)))
        return loss.value, g, out

    def train_step(self, a, target, lr):
        """One Adam step; returns the loss before it."""
        import torch
        out = torch.empty_like(target)
        loss = ctypes.c_double()
        self._check(load().spgpe_fno_train_step(self._h, ctypes.c_void_p(self._dev(a, self.cin)),
                                                ctypes.c_void_p(self._dev(target, self.cout)), int(a.shape[0]),
                                                int(a.shape[2]), ctypes.c_void_p(out.data_ptr()), float(lr),
                                                ctypes.byref(loss)))
        return loss.value


# --------------------------------------------------------- convenience class

class Context:
    """One solver context: an nx x ny grid (optionally a batch of instances).

    Spinors are ``(2, ny, nx)`` or ``(ninst, 2, ny, nx)`` complex arrays:
    torch CUDA tensors (complex64 for ``dtype="c64"``, complex128 for
    ``"c128"``), stepped in place on this context's stream, or numpy arrays
    on the host, which the library copies in, steps and copies back.
    """

    def __init__(self, nx, ny, xmax, ymax, dtype="c64", ninst=1, stream=None, classes=None):
        self.dtype = {"c64": SPGPE_C64, "c128": SPGPE_C128}[dtype]
        self.np_dtype = np.complex64 if self.dtype == SPGPE_C64 else np.complex128
        self.stream = stream
        s = 0
        if stream is not None:
            s = int(getattr(stream, "cuda_stream", stream))
        self.classes = None
        if classes is not None:
            # multi-size batch: spinors are flat buffers; see class_views()
            self.classes = [(int(a), int(b), int(n), float(xm), float(ym)) for a, b, n, xm, ym in classes]
            self.nx = self.ny = None
            self.ninst = sum(c[2] for c in self.classes)
            self._ctx = spgpe_init_multi(self.classes, self.dtype, s)
            return
        self.nx, self.ny, self.ninst = int(nx), int(ny), int(ninst)
        self._ctx = (spgpe_init_batch(nx, ny, xmax, ymax, ninst, self.dtype, s) if ninst != 1
                     else spgpe_init_grid(nx, ny, xmax, ymax, self.dtype, s))

    @classmethod
    def multi(cls, classes, dtype="c64", stream=None):
        """A batch over several grid sizes: classes = [(nx, ny, ninst, xmax, ymax), ...]."""
        return cls(None, None, None, None, dtype, stream=stream, classes=classes)

    def class_sizes(self):
        """Complex elements of each class in the flat spinor buffer of a multi-size batch."""
        return [n * 2 * b * a for a, b, n, _, _ in self.classes]

    def class_views(self, flat):
        """Views (ninst, 2, ny, nx) of the classes in a flat spinor buffer."""
        out, o = [], 0
        for (a, b, n, _, _), sz in zip(self.classes, self.class_sizes()):
            out.append(flat[o:o + sz].reshape(n, 2, b, a))
            o += sz
        return out

    @property
    def handle(self):
        return self._ctx

    def close(self):
        if self._ctx:
            spgpe_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check_psi(self, psi):
        if self.classes is not None:
            total = sum(self.class_sizes())
            if tuple(psi.shape) != (total,):
                raise ValueError(f"a multi-size batch takes a flat spinor of {total} elements")
        shape = tuple(psi.shape) if self.classes is None else None
        if shape is not None:
            want = (2, self.ny, self.nx) if self.ninst == 1 else (self.ninst, 2, self.ny, self.nx)
            if shape not in (want, (self.ninst, 2, self.ny, self.nx)):
                raise ValueError(f"spinor shape {shape}, expected {want}")
        if isinstance(psi, np.ndarray):
            if psi.dtype != self.np_dtype or not psi.flags.c_contiguous:
                raise ValueError(f"host spinor must be C-contiguous {np.dtype(self.np_dtype).name}")
            return psi.ctypes.data
        import torch  # device memory and streams only
        want_t = torch.complex64 if self.dtype == SPGPE_C64 else torch.complex128
        if psi.dtype != want_t or not psi.is_contiguous() or not psi.is_cuda:
            raise ValueError(f"device spinor must be a contiguous CUDA {want_t} tensor")
        return psi.data_ptr()

    def set_potentials(self, V=None, delta=None, Omega=None, g11=0.0, g22=0.0, g12=0.0, kL=0.0):
        n = self.nx * self.ny
        spgpe_set_potentials(self._ctx, *(None if a is None else _f64(a, n) for a in (V, delta, Omega)),
                             g11, g22, g12, kL)

    def set_potentials_separable(self, inst=-1, Vx=None, Vy=None, delta_x=None, delta_y=None, Omega_x=None,
                                 Omega_y=None, g11=0.0, g22=0.0, g12=0.0, kL=0.0):
        nx, ny = self.nx, self.ny
        if self.classes is not None:
            first = 0
            for a, b, n, _, _ in self.classes:
                if inst == -1 or first <= inst < first + n:
                    nx, ny = a, b
                    break
                first += n
        spgpe_set_potentials_separable(self._ctx, inst, _f64(Vx, nx), _f64(Vy, ny), _f64(delta_x, nx),
                                       _f64(delta_y, ny), _f64(Omega_x, nx), _f64(Omega_y, ny),
                                       g11, g22, g12, kL)

    def step_real(self, psi, dt, nsteps):
        spgpe_step_real(self._ctx, self._check_psi(psi), dt, nsteps)
        return psi

    def step_imag(self, psi, dtau, nsteps, norm_mode=SPGPE_NORM_TOTAL, target=(0.5, 0.5), residual=False,
                  lagged=False):
        mode = norm_mode | (SPGPE_IMAG_LAGGED if lagged else 0)
        return spgpe_step_imag(self._ctx, self._check_psi(psi), dtau, nsteps, mode, target,
                               residual, self.ninst)

    def relax(self, psi, dtau, tol, max_steps, check_every=200, norm_mode=SPGPE_NORM_TOTAL, target=(0.5, 0.5),
              ladder=False, handoff=0.0, give_up=False, lagged=False):
        flags = ((SPGPE_RELAX_LADDER if ladder else 0) | (SPGPE_RELAX_GIVE_UP if give_up else 0) |
                 (SPGPE_RELAX_LAGGED if lagged else 0))
        return spgpe_relax(self._ctx, self._check_psi(psi), dtau, tol, max_steps, check_every, norm_mode, target,
                           flags, handoff, self.ninst)

    def autotune(self, psi, dt):
        return spgpe_autotune(self._ctx, self._check_psi(psi), dt, 1 if self.classes is None else len(self.classes))

    def cufft_step_real(self, psi, dt, nsteps):
        spgpe_cufft_step_real(self._ctx, self._check_psi(psi), dt, nsteps)
        return psi

    def observables(self, psi):
        return spgpe_observables(self._ctx, self._check_psi(psi), self.ninst)

    def add_noise(self, psi, sigma, seed):
        spgpe_add_noise(self._ctx, self._check_psi(psi), sigma, seed)
        return psi

    def energy(self, psi):
        return spgpe_energy(self._ctx, self._check_psi(psi), self.ninst)

    def norm(self, psi):
        return spgpe_norm(self._ctx, self._check_psi(psi), self.ninst)

    def sync(self):
        spgpe_sync(self._ctx)

    def wait_probe(self, cycles=1 << 20):
        """Status code of the bounded-wait failure probe (SPGPE_ETIMEOUT expected)."""
        return spgpe_wait_probe(self._ctx, cycles)

    def last_launches(self):
        return spgpe_last_launches(self._ctx)

    def set_timing(self, enable=True):
        spgpe_set_timing(self._ctx, enable)

    def timing(self):
        return spgpe_timing(self._ctx)
