"""ctypes binding of libspgpe.so: the C ABI of include/spgpe.h, names unchanged.

Argument marshalling only; every step of the method runs in the library's
CUDA kernels.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspgpe.so")

SPGPE_C64, SPGPE_C128 = 1, 2
SPGPE_NORM_TOTAL, SPGPE_NORM_PER_COMPONENT = 0, 1
SPGPE_IMAG_LAGGED = 4
SPGPE_RELAX_LADDER, SPGPE_RELAX_GIVE_UP, SPGPE_RELAX_LAGGED = 1, 2, 4
SPGPE_OK, SPGPE_ETIMEOUT = 0, -5
STATUS = {0: "SPGPE_OK", -1: "SPGPE_EINVAL", -2: "SPGPE_ENOMEM", -3: "SPGPE_ECUDA",
          -4: "SPGPE_ENONFINITE", -5: "SPGPE_ETIMEOUT", -6: "SPGPE_ESTATE", -7: "SPGPE_EBOUNDS"}

# Every entry point declared in include/spgpe.h, with its ctypes signature.
_P, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "spgpe_init_grid": (_I, [ctypes.POINTER(_P), _I, _I, _D, _D, _I, _P]),
    "spgpe_init_batch": (_I, [ctypes.POINTER(_P), _I, _I, _D, _D, _I, _I, _P]),
    "spgpe_init_multi": (_I, [ctypes.POINTER(_P), _I, _P, _P, _P, _P, _P, _I, _P]),
    "spgpe_set_potentials": (_I, [_P, _P, _P, _P, _D, _D, _D, _D]),
    "spgpe_set_potentials_separable": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _D, _D, _D, _D]),
    "spgpe_step_real": (_I, [_P, _P, _D, _I]),
    "spgpe_step_imag": (_I, [_P, _P, _D, _I, _I, _P, _P]),
    "spgpe_energy": (_I, [_P, _P, _P]),
    "spgpe_norm": (_I, [_P, _P, _P]),
    "spgpe_sync": (_I, [_P]),
    "spgpe_wait_probe": (_I, [_P, ctypes.c_longlong]),
    "spgpe_cufft_step_real": (_I, [_P, _P, _D, _I]),
    "spgpe_destroy": (None, [_P]),
    "spgpe_last_error": (ctypes.c_char_p, [_P]),
    "spgpe_version": (_I, []),
    "spgpe_last_launches": (_I, [_P]),
    "spgpe_set_timing": (_I, [_P, _I]),
    "spgpe_timing": (_I, [_P, _P, _P]),
    "spgpe_norm_noalloc": (_I, [_P, _I, _I, _I, _D, _D, _I, _P, _P]),
    "spgpe_relax": (_I, [_P, _P, _D, _D, _I, _I, _I, _P, _I, _D, _P, _P]),
    "spgpe_autotune": (_I, [_P, _P, _D, _P, _P]),
    "spgpe_observables": (_I, [_P, _P, _P]),
    "spgpe_fno_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _I, _I, ctypes.c_ulonglong, _P]),
    "spgpe_fno_num_params": (ctypes.c_long, [_P]),
    "spgpe_fno_get_params": (_I, [_P, _P]),
    "spgpe_fno_set_params": (_I, [_P, _P]),
    "spgpe_fno_forward": (_I, [_P, _P, _I, _I, _P]),
    "spgpe_fno_gradient": (_I, [_P, _P, _P, _I, _I, _P, _P, _P]),
    "spgpe_fno_train_step": (_I, [_P, _P, _P, _I, _I, _P, _D, _P]),
    "spgpe_fno_destroy": (None, [_P]),
    "spgpe_fno_last_error": (ctypes.c_char_p, [_P]),
    "spgpe_add_noise": (_I, [_P, _P, _D, ctypes.c_ulonglong]),
    "spgpe_probe_ceilings": (_I, [_P, _I]),
}
PROBE_SIZES_MIB = [16, 32, 64, 96, 128, 160, 192, 256, 512]
NKINDS = 10
KIND_NAMES = ["row_real_open", "row_real_fused", "row_real_close", "col_real", "row_imag_open",
              "row_imag_B", "row_imag_A", "row_imag_rescale", "col_imag", "row_imag_lagged"]

_lock = threading.Lock()
_lib = None


class SpgpeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def load(path: str | None = None):
    """Load libspgpe.so (raises if it is missing: there is no CPU fallback).
    SPGPE_LIBRARY names another build of the same library (the bounds-checked
    one, libspgpe_bounds.so) for a process that wants it."""
    global _lib
    if path is None:
        path = os.environ.get("SPGPE_LIBRARY") or LIB_PATH
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libspgpe.so not built ({path}); run "
                                   "paper_2010_15069_gb300.build.build() on a machine with nvcc")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def check(code: int, ctx=None) -> int:
    if code != 0:
        msg = load().spgpe_last_error(ctx)
        raise SpgpeError(code, msg.decode() if msg else "")
    return code
