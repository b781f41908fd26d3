"""Relaxation to a residual tolerance (spgpe_relax), plain and with the
complex64 -> complex128 precision ladder, through the C ABI.

The imaginary-time map of Sec. 3.2 has one fixed point for these couplings
(miscible, Raman-coupled, no spin-orbit term, so every mode is gapped), so
both routes must end on the same state: the plain complex128 route is checked
against the FP64 oracle run for the same number of steps, and the ladder
against the plain route, within the residual over the gap.
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


def small_problem():
    return inputs.problem(64, 64, 8.0, 8.0, Omega=0.5, delta_slope=0.1, g11=50.0, g22=40.0, g12=20.0)


def ctx(p, dtype, ninst=1):
    g = p.grid
    c = sp.Context(g.nx, g.ny, g.xmax, g.ymax, dtype, ninst)
    c.set_potentials_separable(-1, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    return c


DTAU, TOL = 1e-2, 1e-8


def test_plain_relaxation_reaches_tol_and_matches_oracle(orc):
    p = small_problem()
    psi0 = inputs.gaussian_spinor(p.grid, seed=31)
    with ctx(p, "c128") as c:
        t = torch.from_numpy(psi0.copy()).cuda()
        res, (s64, s) = c.relax(t, DTAU, TOL, 20000, check_every=100)
        got = t.cpu().numpy()
    assert s64 == 0 and 0 < s < 20000 and s % 100 == 0
    assert res[0] <= TOL
    g = p.grid
    m = orc.Model(g.nx, g.ny, g.xmax, g.ymax, V=p.V, delta=p.delta, Omega=p.Omega,
                  g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    ref = m.step(psi0, DTAU, s, imag=True, norm_mode=sp.SPGPE_NORM_TOTAL)
    assert np.abs(got - ref).max() < 1e-11


@pytest.mark.parametrize("handoff", [0.0, 1e-3])
def test_ladder_ends_on_the_plain_fixed_point(handoff):
    p = small_problem()
    psi0 = np.stack([inputs.vortex_spinor(p.grid, n_vortices=6, radius=3.0, seed=40 + i) for i in range(3)])
    with ctx(p, "c128", ninst=3) as c:
        a = torch.from_numpy(psi0.copy()).cuda()
        b = a.clone()
        ra, (sa64, sa) = c.relax(a, DTAU, TOL, 40000, check_every=100)
        rb, (sb64, sb) = c.relax(b, DTAU, TOL, 40000, check_every=100, ladder=True, handoff=handoff)
        ea, eb = c.energy(a)[:, 0], c.energy(b)[:, 0]
        nb = c.norm(b).sum(axis=1)
    assert (ra <= TOL).all() and (rb <= TOL).all()
    assert sa64 == 0 and sb64 > 0 and sb > 0           # part of the way in complex64, the rest in complex128
    assert np.abs(a.cpu().numpy() - b.cpu().numpy()).max() < 1e-5
    assert np.allclose(eb, ea, rtol=1e-10, atol=0)
    assert np.allclose(nb, 1.0, rtol=1e-12)


def test_relax_rejects_bad_arguments():
    p = small_problem()
    with ctx(p, "c64") as c:
        t = torch.zeros((2, 64, 64), dtype=torch.complex64, device="cuda")
        for kw in (dict(tol=0.0), dict(max_steps=0), dict(check_every=0)):
            args = dict(dtau=DTAU, tol=TOL, max_steps=10, check_every=5)
            args.update(kw)
            with pytest.raises(sp.SpgpeError, match="EINVAL"):
                c.relax(t, **args)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batched_relaxation_freezes_each_instance_where_it_converged_alone(dtype):
    """Instances converge after different numbers of chunks; a converged one
    is frozen while the rest go on, so every instance of the batch ends with
    the bits of its own single-instance relaxation."""
    p = small_problem()
    npt = np.complex64 if dtype == "c64" else np.complex128
    tol = 1e-8 if dtype == "c128" else 1e-4
    psi0 = np.stack([inputs.vortex_spinor(p.grid, n_vortices=2 + 3 * i, radius=3.0, seed=50 + i)
                     for i in range(3)]).astype(npt)
    with ctx(p, dtype, ninst=3) as c:
        t = torch.from_numpy(psi0.copy()).cuda()
        res, (_, steps) = c.relax(t, DTAU, tol, 40000, check_every=100)
        got = t.cpu().numpy()
    alone = []
    for i in range(3):
        with ctx(p, dtype) as c1:
            t1 = torch.from_numpy(psi0[i].copy()).cuda()
            r1, (_, s1) = c1.relax(t1, DTAU, tol, 40000, check_every=100)
            alone.append((t1.cpu().numpy(), r1[0], s1))
    assert steps == max(a[2] for a in alone)
    for i in range(3):
        assert res[i] == alone[i][1]
        assert np.array_equal(got[i], alone[i][0]), i


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_relaxation_on_a_stream_replays_chunk_graphs_with_the_same_bits(dtype):
    """On a stream of its own the relaxation captures one chunk in a CUDA graph
    and replays it; on the legacy default stream (which cannot be captured) it
    launches directly.  Both give the same bits and launch counts."""
    p = small_problem()
    npt = np.complex64 if dtype == "c64" else np.complex128
    tol = 1e-8 if dtype == "c128" else 1e-4
    psi0 = np.stack([inputs.vortex_spinor(p.grid, n_vortices=3 + i, radius=3.0, seed=70 + i)
                     for i in range(2)]).astype(npt)
    out = []
    for stream in (None, torch.cuda.Stream()):
        g = p.grid
        with sp.Context(g.nx, g.ny, g.xmax, g.ymax, dtype, 2, stream=stream) as c:
            c.set_potentials_separable(-1, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
            t = torch.from_numpy(psi0.copy()).cuda()
            torch.cuda.synchronize()
            res, steps = c.relax(t, DTAU, tol, 40000, check_every=100, ladder=True)
            torch.cuda.synchronize()
            out.append((t.cpu().numpy(), res, steps, c.last_launches()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2] and out[0][3] == out[1][3]
