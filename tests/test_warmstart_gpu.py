"""What the learned warm start gains: an FNO trained on ground states the
library computed proposes initial spinors for held-out parameter sets, and the
plain imaginary-time relaxation (which decides the result) needs fewer steps
from them than from the vortex-seeded spinors of Sec. 6.
"""
import numpy as np
import pytest

import paper_2010_15069_gb300 as sp
from paper_2010_15069_gb300 import inputs, warmstart

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2010_15069_gb300 import build
    build.build()
    sp.load()


N, BOX, DTAU = 64, 8.0, 5e-3


def sweep(k, seed):
    prm = inputs.sweep_params(k, seed=seed)
    return [dict(q, g=min(q["g"], 800.0), g12=q["g12"] * min(q["g"], 800.0) / q["g"]) for q in prm]


def ctx(prms, dtype):
    c = sp.Context(N, N, BOX, BOX, dtype, ninst=len(prms))
    for i, q in enumerate(prms):
        p = inputs.problem(N, N, BOX, BOX, Omega=q["Omega"], delta_slope=q["delta_slope"], g11=q["g"], g22=q["g"],
                           g12=q["g12"], kL=1.0)
        c.set_potentials_separable(i, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    return c


def cold(grid, k, seed0):
    return np.stack([inputs.vortex_spinor(grid, n_vortices=20, radius=3.0, seed=seed0 + i) for i in range(k)])


def test_trained_fno_warm_start_saves_relaxation_steps():
    grid = inputs.Grid(N, N, BOX, BOX)
    train, test = sweep(32, 21), sweep(8, 77)
    # training targets: ground states from the batched complex64 relaxation
    with ctx(train, "c64") as c:
        t = torch.from_numpy(cold(grid, 32, 500).astype(np.complex64)).cuda()
        c.relax(t, DTAU, 1e-4, 20000, check_every=200, give_up=True)
        gs = t.cpu().numpy().astype(np.complex128)
    feats = lambda prms: np.stack([warmstart.features(grid, q["g"], q["g12"], q["Omega"], q["delta_slope"])
                                   for q in prms])
    a = torch.from_numpy(feats(train)).cuda()
    y = torch.from_numpy(np.stack([warmstart.to_channels(s) for s in gs])).cuda()
    with sp.FNO(warmstart.CIN, warmstart.COUT, width=32, modes=12, layers=4, hidden=64, seed=1) as f:
        losses = []
        for it in range(1500):
            idx = torch.from_numpy(np.random.default_rng(it).choice(32, 8, replace=False)).cuda()
            losses.append(f.train_step(a[idx].contiguous(), y[idx].contiguous(), 2e-3))
        pred = f.forward(torch.from_numpy(feats(test)).cuda()).cpu().numpy()
    assert np.mean(losses[-20:]) < 1e-2
    warm = np.stack([warmstart.from_channels(p) for p in pred])
    starts = {"cold": cold(grid, 8, 900), "warm": warm}
    # residual of the held-out batch after 4000 complex128 steps (geometric mean)
    after = {}
    for name, psi0 in starts.items():
        with ctx(test, "c128") as c:
            tt = torch.from_numpy(np.ascontiguousarray(psi0)).cuda()
            c.step_imag(tt, DTAU, 3999)
            after[name] = float(np.exp(np.log(c.step_imag(tt, DTAU, 1, residual=True)).mean()))
    assert after["warm"] < 0.5 * after["cold"], after
    # instances that reach residual 1e-3 within 20000 steps
    reached = {}
    for name, psi0 in starts.items():
        with ctx(test, "c128") as c:
            tt = torch.from_numpy(np.ascontiguousarray(psi0)).cuda()
            res, _ = c.relax(tt, DTAU, 1e-3, 20000, check_every=100)
            reached[name] = int((res <= 1e-3).sum())
    assert reached["warm"] > reached["cold"], reached


def test_warm_start_trained_at_256_helps_at_512():
    """The resolution change of the warm-start protocol: a network trained on
    ground states the solver computed at 256^2 (box [-12, 12]^2, sweep
    generator) proposes the initial spinors of held-out parameter sets at
    512^2 on the same box; the imaginary-time relaxation from them is ahead
    of the relaxation from vortex-seeded spinors."""
    L, n0, n1 = 12.0, 256, 512
    g0, g1 = inputs.Grid(n0, n0, L, L), inputs.Grid(n1, n1, L, L)
    train, test = sweep(48, 31), sweep(8, 97)

    def sctx(prms, n, dtype):
        c = sp.Context(n, n, L, L, dtype, ninst=len(prms))
        for i, q in enumerate(prms):
            p = inputs.problem(n, n, L, L, Omega=q["Omega"], delta_slope=q["delta_slope"], g11=q["g"], g22=q["g"],
                               g12=q["g12"], kL=1.0)
            c.set_potentials_separable(i, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
        return c

    with sctx(train, n0, "c64") as c:
        t = torch.from_numpy(np.stack([inputs.vortex_spinor(g0, n_vortices=20, radius=5.0, seed=600 + i)
                                       for i in range(48)]).astype(np.complex64)).cuda()
        c.relax(t, DTAU, 2e-3, 20000, check_every=250, give_up=True, lagged=True)
        gs = t.cpu().numpy().astype(np.complex128)
    feats = lambda prms, g: np.stack([warmstart.features(g, q["g"], q["g12"], q["Omega"], q["delta_slope"])
                                      for q in prms])
    a = torch.from_numpy(feats(train, g0)).cuda()
    y = torch.from_numpy(np.stack([warmstart.to_channels(s) for s in gs])).cuda()
    with sp.FNO(warmstart.CIN, warmstart.COUT, width=32, modes=12, layers=4, hidden=64, seed=3) as f:
        for it in range(1500):
            idx = torch.from_numpy(np.random.default_rng(it).choice(48, 8, replace=False)).cuda()
            f.train_step(a[idx].contiguous(), y[idx].contiguous(), 2e-3)
        pred = f.forward(torch.from_numpy(feats(test, g1)).cuda()).cpu().numpy()
    starts = {"cold": np.stack([inputs.vortex_spinor(g1, n_vortices=20, radius=5.0, seed=900 + i) for i in range(8)]),
              "warm": np.stack([warmstart.from_channels(p) for p in pred])}
    after = {}
    for name, psi0 in starts.items():
        with sctx(test, n1, "c64") as c:
            tt = torch.from_numpy(np.ascontiguousarray(psi0).astype(np.complex64)).cuda()
            c.step_imag(tt, DTAU, 1999, lagged=True)
            after[name] = float(np.exp(np.log(c.step_imag(tt, DTAU, 1, residual=True)).mean()))
    assert after["warm"] < 0.5 * after["cold"], after
