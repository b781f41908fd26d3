"""The bounds-checked build (libspgpe_bounds.so, -DSPGPE_BOUNDS) against the
release build, bit for bit.

The stand-in for a memory checker is a build whose
kernels check every global index of the step passes (spinor loads and stores,
the bulk-copy and TMA boxes, the step tables, the atom-number partials)
against its buffer, record an index outside it as SPGPE_EBOUNDS and skip the
access.  The same protocol (real-time steps, exact and lagged imaginary-time
steps, energies and atom numbers) runs through both builds, each in a process
of its own, on small and ragged grids and on the shapes that select the other
pass variants (warp-local columns, block-wide rows, tall columns), with the
plain and the persistent passes, in both precisions: no index may fall
outside its buffer, and the results must be the same bits.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CASES = [(8, 8), (16, 16), (32, 64), (64, 32), (256, 256), (512, 32), (16, 2048)]
SCHEDULES = {"persistent": "2", "plain": "0"}


def protocol(out_path):
    """Run every case through the library this process loaded; save the results."""
    sys.path.insert(0, ROOT)
    import torch
    import paper_2010_15069_gb300 as sp
    from paper_2010_15069_gb300 import inputs
    res = {}
    for sched, env in SCHEDULES.items():
        os.environ["SPGPE_PERSISTENT"] = env
        for nx, ny in CASES:
            for dtype, npt in (("c64", np.complex64), ("c128", np.complex128)):
                p = inputs.problem(nx, ny, max(1.0, 0.05 * nx), max(1.0, 0.05 * ny), Omega=1.3, delta_slope=0.4,
                                   g11=40.0, g22=35.0, g12=30.0, kL=0.7)
                psi0 = np.stack([inputs.gaussian_spinor(p.grid, width=0.4 * min(p.grid.xmax, p.grid.ymax),
                                                        noise=0.2, seed=nx + ny + i) for i in range(2)])
                g = p.grid
                with sp.Context(g.nx, g.ny, g.xmax, g.ymax, dtype, ninst=2) as c:
                    c.set_potentials_separable(-1, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
                    t = torch.from_numpy(psi0.astype(npt)).cuda()
                    c.step_real(t, 2e-3, 5)
                    c.step_imag(t, 2e-3, 4, sp.SPGPE_NORM_PER_COMPONENT, (0.6, 0.4))
                    c.step_imag(t, 2e-3, 5, lagged=True)
                    c.sync()
                    e = c.energy(t)
                    n = c.norm(t)
                    key = f"{sched}_{nx}x{ny}_{dtype}"
                    res[key + "_psi"] = t.cpu().numpy()
                    res[key + "_energy"] = e
                    res[key + "_norm"] = n
    np.savez(out_path, **res)


def run(lib, out):
    env = dict(os.environ)
    env.pop("SPGPE_PERSISTENT", None)
    env.pop("SPGPE_COLPASS", None)
    if lib:
        env["SPGPE_LIBRARY"] = lib
    else:
        env.pop("SPGPE_LIBRARY", None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), str(out)], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]


@pytest.mark.gpu
def test_bounds_checked_build_matches_release_bit_for_bit(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():  # pragma: no cover
        pytest.skip("CUDA not available")
    sys.path.insert(0, ROOT)
    from paper_2010_15069_gb300 import build
    build.build()
    lib_b = build.build(bounds=True)
    rel_out, bnd_out = tmp_path / "release.npz", tmp_path / "bounds.npz"
    run(None, rel_out)
    run(lib_b, bnd_out)   # an SPGPE_EBOUNDS raised there fails the run
    a, b = np.load(rel_out), np.load(bnd_out)
    assert sorted(a.files) == sorted(b.files) and len(a.files) == 3 * 2 * len(CASES) * len(SCHEDULES)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k


if __name__ == "__main__":
    protocol(sys.argv[1])
