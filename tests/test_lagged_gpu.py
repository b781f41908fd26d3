"""The lagged renormalisation of imaginary time (SPGPE_IMAG_LAGGED,
SPGPE_RELAX_LAGGED) through the C ABI.

Sec. 3.2 renormalises after every step S(dtau).  The lagged schedule opens
step n+1 on the closing result of step n scaled by the previous step's scale
and corrects the linear part in the column pass, so only the densities seen
by the opening D lag behind.  A stationary state of the exact map is a
stationary state of the lagged one, so both relax to the same ground state:
checked against the exact relaxation and against the FP64 oracle (one oracle
step from the lagged result moves it by no more than the tolerance), with
mixing, detuning, spin-orbit and unequal couplings on.  The transient differs
from the exact one by O(dtau g rho (s_n^2/s_{n-1}^2 - 1)); the first boundary
and the end of every call are exact, so a call returns a normalised state,
and calls of one or two steps give the exact bits.
"""
import numpy as np
import pytest

import paper_2010_15069_gb300 as sp
from paper_2010_15069_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

NPT = {"c64": np.complex64, "c128": np.complex128}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2010_15069_gb300 import build
    build.build()
    sp.load()


def problem(nx=64, ny=64):
    return inputs.problem(nx, ny, 8.0, 8.0, Omega=1.2, delta_slope=0.2, g11=60.0, g22=50.0, g12=30.0, kL=0.6)


def ctx(p, dtype, ninst=1, stream=None):
    g = p.grid
    c = sp.Context(g.nx, g.ny, g.xmax, g.ymax, dtype, ninst, stream=stream)
    c.set_potentials_separable(-1, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    return c


def model(orc, p):
    g = p.grid
    return orc.Model(g.nx, g.ny, g.xmax, g.ymax, V=p.V, delta=p.delta, Omega=p.Omega,
                     g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)


DTAU = 5e-3


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_one_and_two_steps_are_exact(dtype):
    """No boundary of a one- or two-step call is lagged: the same bits as the
    exact schedule."""
    p = problem()
    psi0 = inputs.vortex_spinor(p.grid, n_vortices=4, radius=3.0, seed=5).astype(NPT[dtype])
    with ctx(p, dtype) as c:
        for n in (1, 2):
            a = torch.from_numpy(psi0.copy()).cuda()
            b = a.clone()
            c.step_imag(a, DTAU, n, sp.SPGPE_NORM_PER_COMPONENT, (0.6, 0.4))
            c.step_imag(b, DTAU, n, sp.SPGPE_NORM_PER_COMPONENT, (0.6, 0.4), lagged=True)
            assert torch.equal(a, b), n


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("mode", [sp.SPGPE_NORM_TOTAL, sp.SPGPE_NORM_PER_COMPONENT])
def test_transient_close_to_exact_and_normalised(orc, dtype, mode):
    """40 lagged steps from a vortex-seeded state: two passes per step after the
    first boundary, a normalised result, and a state close to the exact
    schedule's (and to the oracle's, which is exact) at the size the lag
    allows: O(dtau g rho (s_n^2 / s_{n-1}^2 - 1)) per step."""
    p = problem()
    psi0 = inputs.vortex_spinor(p.grid, n_vortices=6, radius=3.0, seed=9)
    n = 40
    ref = model(orc, p).step(psi0, DTAU, n, imag=True, norm_mode=mode, target=(0.6, 0.4))
    with ctx(p, dtype) as c:
        t = torch.from_numpy(psi0.astype(NPT[dtype])).cuda()
        c.step_imag(t, DTAU, n, mode, (0.6, 0.4), lagged=True)
        assert c.last_launches() == 2 * n + 3
        nrm = c.norm(t)[0]
        got = t.cpu().numpy().astype(np.complex128)
    rt = 1e-12 if dtype == "c128" else 1e-6
    if mode == sp.SPGPE_NORM_PER_COMPONENT:
        assert np.allclose(nrm, (0.6, 0.4), atol=rt, rtol=0)
    else:
        assert abs(nrm.sum() - 1.0) < rt
    d = np.abs(got - ref).max()
    assert 0 < d < 2e-3 * np.abs(ref).max(), d


@pytest.mark.parametrize("mode", [sp.SPGPE_NORM_TOTAL, sp.SPGPE_NORM_PER_COMPONENT])
def test_lagged_relaxation_ends_on_the_exact_fixed_point(orc, mode):
    """complex128: the lagged and the exact relaxation to residual 1e-10 end on
    the same state up to the global phase (a symmetry of the map, which the
    two transients rotate differently), within the residual over the gap, with
    the same energy, and one exact oracle step from the lagged result stays
    within the tolerance."""
    p = problem()
    psi0 = np.stack([inputs.gaussian_spinor(p.grid, width=1.5, noise=0.1, seed=20 + i, center=(0.7, -0.4 * i),
                                            momentum=(0.5, 0.2)) for i in range(2)])
    tol, dtau = 1e-10, 1e-2
    with ctx(p, "c128", ninst=2) as c:
        a = torch.from_numpy(psi0.copy()).cuda()
        b = a.clone()
        ra, _ = c.relax(a, dtau, tol, 60000, check_every=100, norm_mode=mode, target=(0.6, 0.4))
        rb, (_, sb) = c.relax(b, dtau, tol, 60000, check_every=100, norm_mode=mode, target=(0.6, 0.4),
                              lagged=True)
        ea, eb = c.energy(a)[:, 0], c.energy(b)[:, 0]
        ga, gb = a.cpu().numpy(), b.cpu().numpy()
    assert (ra <= tol).all() and (rb <= tol).all() and sb > 0
    for i in range(2):
        ph = np.vdot(gb[i], ga[i])
        assert np.abs(ga[i] - gb[i] * ph / abs(ph)).max() < 1e-8, i
    assert np.allclose(eb, ea, rtol=1e-12, atol=0)
    m = model(orc, p)
    for i in range(2):
        _, r_or = m.step(gb[i], dtau, 1, imag=True, norm_mode=mode, target=(0.6, 0.4), residual=True)
        assert r_or < 3 * tol, (i, r_or)


def test_ladder_with_lagged_stages():
    """The complex64 -> complex128 ladder with both stages lagged ends on the
    fixed point of the exact complex128 relaxation (miscible, Raman-coupled, no
    spin-orbit term: every mode gapped; vortex-seeded starts)."""
    p = inputs.problem(64, 64, 8.0, 8.0, Omega=0.5, delta_slope=0.1, g11=50.0, g22=40.0, g12=20.0)
    psi0 = np.stack([inputs.vortex_spinor(p.grid, n_vortices=6, radius=3.0, seed=40 + i) for i in range(3)])
    tol, dtau = 1e-8, 1e-2
    with ctx(p, "c128", ninst=3) as c:
        a = torch.from_numpy(psi0.copy()).cuda()
        b = a.clone()
        ra, _ = c.relax(a, dtau, tol, 60000, check_every=100)
        rb, (s64, s) = c.relax(b, dtau, tol, 60000, check_every=100, ladder=True, lagged=True)
        ea, eb = c.energy(a)[:, 0], c.energy(b)[:, 0]
        nb = c.norm(b).sum(axis=1)
    assert (ra <= tol).all() and (rb <= tol).all() and s64 > 0 and s > 0
    ga, gb = a.cpu().numpy(), b.cpu().numpy()
    for i in range(3):  # up to the global phase
        ph = np.vdot(gb[i], ga[i])
        assert np.abs(ga[i] - gb[i] * ph / abs(ph)).max() < 1e-5, i
    assert np.allclose(eb, ea, rtol=1e-10, atol=0)
    assert np.allclose(nb, 1.0, rtol=1e-12)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_host_chunks_multi_size_and_graph_replay_keep_the_bits(dtype):
    """The lagged schedule through the other paths: a host spinor batch (in
    chunks of instances), a multi-size batch (each instance as in a
    single-size context) and relaxation chunks replayed from a CUDA graph on a
    stream of its own (as launched directly on the legacy stream)."""
    p = problem()
    npt = NPT[dtype]
    psi0 = np.stack([inputs.vortex_spinor(p.grid, n_vortices=3 + i, radius=3.0, seed=40 + i)
                     for i in range(5)]).astype(npt)
    with ctx(p, dtype, ninst=5) as c:
        t = torch.from_numpy(psi0.copy()).cuda()
        c.step_imag(t, DTAU, 17, lagged=True)
        h = psi0.copy()
        c.step_imag(h, DTAU, 17, lagged=True)
        dev = t.cpu().numpy()
        assert np.array_equal(dev, h)
    q = problem(32, 128)
    psi_q = inputs.vortex_spinor(q.grid, n_vortices=3, radius=2.0, seed=47).astype(npt)
    classes = [(64, 64, 5, 8.0, 8.0), (32, 128, 1, 8.0, 8.0)]
    with sp.Context.multi(classes, dtype) as c:
        for k in range(5):
            c.set_potentials_separable(k, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
        c.set_potentials_separable(5, **q.separable, g11=q.g11, g22=q.g22, g12=q.g12, kL=q.kL)
        flat = torch.from_numpy(np.concatenate([psi0.ravel(), psi_q.ravel()])).cuda()
        c.step_imag(flat, DTAU, 17, lagged=True)
        v = c.class_views(flat)
        assert np.array_equal(v[0].cpu().numpy(), dev)
    out = []
    for stream in (None, torch.cuda.Stream()):
        with ctx(p, dtype, ninst=2, stream=stream) as c:
            t = torch.from_numpy(psi0[:2].copy()).cuda()
            torch.cuda.synchronize()
            res, steps = c.relax(t, DTAU, 1e-8 if dtype == "c128" else 1e-4, 4000, check_every=100, lagged=True)
            torch.cuda.synchronize()
            out.append((t.cpu().numpy(), res, steps, c.last_launches()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2] and out[0][3] == out[1][3]
