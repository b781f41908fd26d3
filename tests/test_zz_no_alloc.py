"""spgpe_norm_noalloc, the allocation-free atom-number entry point, against spgpe_norm.

Some callers cannot let a library call cudaMalloc (applications that own all
device memory through their own pool, or run under a fixed memory budget);
this entry point keeps its partial sums in device memory that is part of the
library.  Checked through the C ABI, twice in a row (the shared scratch keeps
the previous call's contents), against the context-based spgpe_norm within
the tolerances of the other parity tests.  This file sorts last so that a run
stopping at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import paper_2010_15069_gb300 as sp
from paper_2010_15069_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)


@pytest.mark.parametrize("dtype,code,rtol", [("c128", sp.SPGPE_C128, 1e-12), ("c64", sp.SPGPE_C64, 2e-6)])
def test_norm_noalloc_matches_context_norm_on_consecutive_calls(dtype, code, rtol):
    from paper_2010_15069_gb300 import build
    build.build()
    lib = _lib.load()
    nx, ny, ninst, L = 128, 64, 3, 8.0
    g = inputs.Grid(nx, ny, L, L / 2)
    npt = np.complex64 if dtype == "c64" else np.complex128
    stream = torch.cuda.Stream()
    with sp.Context(nx, ny, L, L / 2, dtype, ninst=ninst, stream=stream) as c:
        for call in range(2):
            psi = np.stack([inputs.vortex_spinor(g, n_vortices=4 + i, radius=2.5, seed=10 * call + i,
                                                 target=(0.3 + 0.1 * i, 0.5 - 0.1 * call)) for i in range(ninst)])
            with torch.cuda.stream(stream):
                t = torch.from_numpy(psi.astype(npt)).cuda()
            stream.synchronize()
            ref = c.norm(t).reshape(-1)
            out = np.zeros(2 * ninst)
            rc = lib.spgpe_norm_noalloc(ctypes.c_void_p(t.data_ptr()), nx, ny, ninst, L, L / 2, code,
                                        ctypes.c_void_p(stream.cuda_stream),
                                        out.ctypes.data_as(ctypes.c_void_p))
            assert rc == 0, sp.spgpe_last_error(None)
            assert np.allclose(out, ref, rtol=rtol, atol=0), (call, out, ref)


def test_norm_noalloc_rejects_sizes_beyond_its_scratch():
    lib = _lib.load()
    t = torch.zeros((2, 8, 8), dtype=torch.complex64, device="cuda")
    out = np.zeros(2 * 300)
    rc = lib.spgpe_norm_noalloc(ctypes.c_void_p(t.data_ptr()), 8, 8, 300, 1.0, 1.0, sp.SPGPE_C64, None,
                                out.ctypes.data_as(ctypes.c_void_p))
    assert rc == -1
