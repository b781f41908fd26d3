"""The C ABI library loads and exports every entry point of include/spgpe.h (no GPU).

Only argument checks that fail before any CUDA call are exercised here.
"""
import ctypes
import os
import re

import pytest

import paper_2010_15069_gb300 as sp
from paper_2010_15069_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "spgpe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spgpe_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_15069_gb300 import build
    build.build()
    return _lib.load()


def test_header_and_binding_agree():
    assert declared_entry_points() == sorted(_lib.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name
    assert sp.spgpe_version() == 100


@pytest.mark.parametrize("nx,ny,xmax,dtype", [(7, 8, 1.0, 1), (8, 8192, 1.0, 1), (8, 8, -1.0, 1),
                                               (8, 8, float("nan"), 1), (8, 8, 1.0, 3), (4, 4, 1.0, 2)])
def test_init_rejects_bad_arguments_before_touching_the_gpu(lib, nx, ny, xmax, dtype):
    ctx = ctypes.c_void_p(123)
    rc = lib.spgpe_init_grid(ctypes.byref(ctx), nx, ny, xmax, 1.0, dtype, None)
    assert rc == -1 and ctx.value is None
    assert sp.spgpe_last_error(None)


def test_calls_on_null_context_are_rejected(lib):
    assert lib.spgpe_step_real(None, None, 0.1, 1) == -1
    assert lib.spgpe_step_imag(None, None, 0.1, 1, 0, None, None) == -1
    assert lib.spgpe_energy(None, None, None) == -1
    assert lib.spgpe_norm(None, None, None) == -1
    assert lib.spgpe_sync(None) == -1
    assert lib.spgpe_wait_probe(None, 1) == -1
    assert lib.spgpe_last_launches(None) == 0
    lib.spgpe_destroy(None)


def test_package_fails_loudly_without_library(tmp_path):
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved
