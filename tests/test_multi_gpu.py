"""Batches over several grid sizes (spgpe_init_multi) through the C ABI.

Each size class runs on its own stream; an instance's arithmetic does not
depend on the batch around it, so every instance of a multi-size batch must
end with the bits of the same instance stepped in a single-size context, and
sampled instances match the FP64 oracle.
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


CLASSES = [(64, 64, 3, 8.0, 8.0), (128, 32, 2, 10.0, 5.0), (32, 128, 1, 4.0, 12.0), (256, 256, 2, 10.0, 10.0)]
NPT = {"c64": np.complex64, "c128": np.complex128}


def instances():
    """(class, local index, problem, spinor) for every instance, sweep-style parameters."""
    out, k = [], 0
    prm = inputs.sweep_params(sum(c[2] for c in CLASSES), seed=11)
    for ci, (nx, ny, n, xm, ym) in enumerate(CLASSES):
        for j in range(n):
            q = prm[k]
            g = min(q["g"], 300.0)
            p = inputs.problem(nx, ny, xm, ym, Omega=q["Omega"], delta_slope=q["delta_slope"], g11=g, g22=0.9 * g,
                               g12=g * q["g12"] / q["g"], kL=0.7)
            psi = inputs.vortex_spinor(p.grid, n_vortices=3, radius=2.0, seed=60 + k)
            out.append((ci, j, p, psi))
            k += 1
    return out


def set_all(c, insts, multi):
    for k, (ci, j, p, _) in enumerate(insts):
        c.set_potentials_separable(k if multi else j, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_multi_size_batch_matches_single_size_contexts(dtype, orc):
    insts = instances()
    npt = NPT[dtype]
    with sp.Context.multi(CLASSES, dtype) as c:
        set_all(c, insts, True)
        flat = torch.from_numpy(np.concatenate([x[3].astype(npt).ravel() for x in insts])).cuda()
        c.step_real(flat, 1e-3, 11)
        c.step_imag(flat, 2e-3, 7, sp.SPGPE_NORM_PER_COMPONENT)
        res = c.step_imag(flat, 2e-3, 5, residual=True)
        e = c.energy(flat)
        nrm = c.norm(flat)
        views = [v.cpu().numpy() for v in c.class_views(flat)]
    k = 0
    for ci, (nx, ny, n, xm, ym) in enumerate(CLASSES):
        mine = [x for x in insts if x[0] == ci]
        with sp.Context(nx, ny, xm, ym, dtype, ninst=n) as s:
            set_all(s, mine, False)
            t = torch.from_numpy(np.stack([x[3] for x in mine]).astype(npt)).cuda()
            s.step_real(t, 1e-3, 11)
            s.step_imag(t, 2e-3, 7, sp.SPGPE_NORM_PER_COMPONENT)
            rs = s.step_imag(t, 2e-3, 5, residual=True)
            es, ns = s.energy(t), s.norm(t)
            ref = t.cpu().numpy()
        assert np.array_equal(views[ci], ref), ci
        assert np.array_equal(res[k:k + n], rs) and np.array_equal(e[k:k + n], es) and np.array_equal(nrm[k:k + n], ns)
        k += n
    # one instance of the widest class against the oracle
    ci, j, p, psi = insts[-1]
    g = p.grid
    m = orc.Model(g.nx, g.ny, g.xmax, g.ymax, V=p.V, delta=p.delta, Omega=p.Omega,
                  g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    want = m.step(psi, 1e-3, 11)
    want = m.step(want, 2e-3, 7, imag=True, norm_mode=sp.SPGPE_NORM_PER_COMPONENT)
    want = m.step(want, 2e-3, 5, imag=True, norm_mode=sp.SPGPE_NORM_TOTAL)
    tol = 1e-11 if dtype == "c128" else 2e-5
    assert np.abs(views[ci][j] - want).max() < tol


def test_multi_size_relaxation_and_host_spinors():
    insts = instances()
    with sp.Context.multi(CLASSES, "c128") as c:
        set_all(c, insts, True)
        host = np.concatenate([x[3].ravel() for x in insts])
        d = torch.from_numpy(host.copy()).cuda()
        c.step_real(host, 1e-3, 4)                  # host spinor: staged for the whole batch
        c.step_real(d, 1e-3, 4)
        assert np.array_equal(d.cpu().numpy(), host)
        res, (s64, s) = c.relax(d, 1e-2, 1e-8, 20000, check_every=100, ladder=True, give_up=True)
        e = c.energy(d)[:, 0]
    assert s64 > 0 and s > 0
    assert np.isfinite(res).all() and np.isfinite(e).all()
    assert (res <= 1e-8).sum() >= len(insts) // 2


@pytest.mark.parametrize("dtype,chunks", [("c64", "1"), ("c64", "3"), ("c128", "8")])
def test_multi_size_host_spinors_go_through_in_chunks_with_the_same_bits(dtype, chunks, monkeypatch):
    """A host spinor of a multi-size batch goes through each class in chunks
    of instances (SPGPE_HOST_CHUNKS per class), copies overlapping the other
    chunks' steps: real time, exact and lagged imaginary time end with the
    bits of the same steps on a device spinor."""
    monkeypatch.setenv("SPGPE_HOST_CHUNKS", chunks)
    insts = instances()
    npt = NPT[dtype]
    with sp.Context.multi(CLASSES, dtype) as c:
        set_all(c, insts, True)
        host = np.concatenate([x[3].astype(npt).ravel() for x in insts])
        d = torch.from_numpy(host.copy()).cuda()
        for call in (lambda x: c.step_real(x, 1e-3, 5), lambda x: c.step_imag(x, 1e-3, 1),
                     lambda x: c.step_imag(x, 1e-3, 7, sp.SPGPE_NORM_PER_COMPONENT, (0.6, 0.4)),
                     lambda x: c.step_imag(x, 1e-3, 6, lagged=True)):
            call(host)
            call(d)
            assert np.array_equal(d.cpu().numpy(), host)


def test_autotune_picks_a_variant_per_class_and_leaves_psi_alone():
    insts = instances()
    with sp.Context.multi(CLASSES, "c64") as c:
        set_all(c, insts, True)
        flat = torch.from_numpy(np.concatenate([x[3].astype(np.complex64).ravel() for x in insts])).cuda()
        before = flat.clone()
        choice, ms = c.autotune(flat, 1e-3)
        assert torch.equal(flat, before)
        assert choice.shape == (len(CLASSES),) and (choice >= 0).all()
        for (nx, ny, *_), v in zip(CLASSES, choice):
            # bit 0 the persistent row pass, v >> 1 the column pass: plain, TMA, or
            # (complex64, 256 rows) the warp-local one
            assert v <= (5 if ny == 256 and nx >= 16 else 3), (nx, ny, v)
        assert (ms > 0).all() and np.isfinite(ms).all()
        a = flat.clone()
        c.step_real(a, 1e-3, 9)              # the tuned schedule; real-time variants agree bit for bit
    with sp.Context.multi(CLASSES, "c64") as c:
        set_all(c, insts, True)
        c.step_real(flat, 1e-3, 9)
    assert torch.equal(a, flat)
