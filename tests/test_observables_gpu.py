"""Sec. 6 observables (spgpe_observables) and annealing noise (spgpe_add_noise)
against the FP64 oracle, through the C ABI.

Winding numbers are integers and must agree exactly; the contour radius is a
bin edge and must agree exactly on states whose cumulative atom number is not
within rounding of a bin boundary; the phase-separation parameter agrees to
the rounding of the FP64 sums (of complex64 densities for c64).  The noise is
the same counter-based stream on both sides.
"""
import numpy as np
import pytest

import paper_2010_15069_gb300 as sp
from paper_2010_15069_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2010_15069_gb300 import build
    build.build()
    sp.load()


NPT = {"c64": np.complex64, "c128": np.complex128}


def states(g):
    X, Y = g.mesh()
    env = np.exp(-(X ** 2 + Y ** 2) / 4)

    def core(x0, y0, s):
        z = (X - x0) + 1j * s * (Y - y0)
        return z / np.sqrt(np.abs(z) ** 2 + 0.25)
    return [
        np.stack([env * core(0.5, 0.2, 1) * core(-0.4, -0.6, 1), env * core(0.1, 0.3, -1)]),
        np.stack([np.exp(-((X - 0.8) ** 2 + Y ** 2) / 2), np.exp(-((X + 0.8) ** 2 + Y ** 2) / 2)]).astype(complex),
        inputs.vortex_spinor(g, n_vortices=8, radius=2.0, seed=91),
    ]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("nx,ny,L", [(64, 64, 8.0), (128, 64, 8.0), (256, 256, 10.0)])
def test_observables_match_oracle(orc, dtype, nx, ny, L):
    g = inputs.Grid(nx, ny, L, L)
    sts = [s.astype(NPT[dtype]) for s in states(g)]
    with sp.Context(nx, ny, L, L, dtype, ninst=len(sts)) as c:
        got = c.observables(torch.from_numpy(np.stack(sts)).cuda())
    m = orc.Model(nx, ny, L, L)
    for k, s in enumerate(sts):
        want = m.observables(s.astype(np.complex128))
        assert got[k, 1] == want[1] and got[k, 2] == want[2], (k, got[k], want)
        assert abs(got[k, 3] - want[3]) <= 0.5 * min(g.dx, g.dy) + 1e-12
        assert abs(got[k, 0] - want[0]) < (1e-12 if dtype == "c128" else 1e-6)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_noise_matches_oracle_per_instance(orc, dtype):
    g = inputs.Grid(64, 32, 6.0, 3.0)
    psi = np.stack([inputs.gaussian_spinor(g, seed=s) for s in range(3)]).astype(NPT[dtype])
    with sp.Context(64, 32, 6.0, 3.0, dtype, ninst=3) as c:
        t = torch.from_numpy(psi.copy()).cuda()
        c.add_noise(t, 0.05, seed=2024)
        got = t.cpu().numpy().astype(np.complex128)
    m = orc.Model(64, 32, 6.0, 3.0)
    for i in range(3):
        want = m.add_noise(psi[i].astype(np.complex128), 0.05, seed=2024, inst=i)
        tol = 1e-15 if dtype == "c128" else 1e-7
        assert np.abs(got[i] - want).max() < tol


def test_ground_state_protocol_with_annealing_and_observables():
    """The Sec. 6 protocol on a small grid: vortex-seeded spinor, a first
    imaginary-time segment annealed with noise now and then, a second without,
    then the observables (finite, integer windings)."""
    p = inputs.problem(128, 128, 10.0, 10.0, Omega=1.0, delta_slope=0.2, g11=100.0, g22=100.0, g12=30.0, kL=1.0)
    g = p.grid
    with sp.Context(g.nx, g.ny, g.xmax, g.ymax, "c64") as c:
        c.set_potentials_separable(-1, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
        t = torch.from_numpy(inputs.vortex_spinor(g, n_vortices=50, radius=4.0, seed=2).astype(np.complex64)).cuda()
        for k in range(5):
            c.step_imag(t, 2e-3, 200)
            c.add_noise(t, 1e-3, seed=100 + k)
        c.step_imag(t, 2e-3, 1000)
        o = c.observables(t)[0]
        n = c.norm(t).sum()
    assert np.isfinite(o).all() and 0.0 <= o[0] <= 1.0 and o[1] == round(o[1]) and o[2] == round(o[2])
    assert abs(n - 1.0) < 1e-5
