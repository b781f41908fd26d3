"""Imaginary time at the sizes the sweep and the 1024^2 ground states run,
against the FP64 oracle element by element (Sec. 3.2: normalise after every
step; Sec. 6: 1024^2 ground states).

Cases: 512^2 and 1024^2 grids with every coupling on (Raman, detuning
gradient, SOC, unequal interactions) in both normalisation modes and both
precisions; rows and columns of 512 to 2048 points through each pass variant
(plain, persistent row + TMA column, warp-local column); one sampled instance
of each size class of a sweep batch of the 64 x 256^2 + 16 x 512^2 +
4 x 1024^2 kind; and the 1024^2 ground-state problem (Omega = 4, delta = 0.2 y,
kL = 2, g = 1000, g12 in {900, 1000, 1100}, 50 seeded vortices, dtau = 1e-3)
for 100 steps.  The oracle references of a module run side by side in a
spawned process pool.

Bars: complex128 within 1e-11 max|dpsi| per 100 steps; complex64 within
1e-4 max|dpsi| and 1e-5 relative energy, with the spinor normalised to one
atom.
"""
import numpy as np
import pytest

import oracle_jobs
import paper_2010_15069_gb300 as sp
from paper_2010_15069_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

NPT = {"c64": np.complex64, "c128": np.complex128}
MODES = (sp.SPGPE_NORM_TOTAL, sp.SPGPE_NORM_PER_COMPONENT)
TARGET = (0.55, 0.45)


@pytest.fixture(scope="module", autouse=True)
def built(orc):
    from paper_2010_15069_gb300 import build
    build.build()
    sp.load()


def to_dev(psi, dtype):
    return torch.from_numpy(np.ascontiguousarray(psi.astype(NPT[dtype]))).cuda()


def to_host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def tol_psi(dtype, n):
    return 1e-11 * max(1.0, n / 100.0) if dtype == "c128" else 1e-4


def tol_energy(dtype):
    return 1e-11 if dtype == "c128" else 1e-5


def sweep_like(nx, ny, box=12.0, g=500.0):
    return inputs.problem(nx, ny, box, box, Omega=3.0, delta_slope=0.6, g11=g, g22=0.9 * g, g12=0.95 * g, kL=1.0)


def ctx_for(p, dtype, ninst=1):
    g = p.grid
    c = sp.Context(g.nx, g.ny, g.xmax, g.ymax, dtype, ninst)
    c.set_potentials_separable(-1, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    return c


# ------------------------------------------------------ oracle references

LARGE = [512, 1024]
LARGE_STEPS, LARGE_DTAU = 60, 5e-3
VARIANT_GRIDS = [(2048, 16), (16, 2048), (1024, 32), (32, 1024), (512, 64), (64, 512), (512, 256)]
VARIANT_STEPS = 40
MULTI = [(256, 256, 3, 12.0, 12.0), (512, 512, 2, 12.0, 12.0), (1024, 1024, 1, 12.0, 12.0)]
MULTI_SAMPLES = (1, 4, 5)
MULTI_STEPS = 40
CONFIG2_G12 = (900.0, 1000.0, 1100.0)
CONFIG2_STEPS = 100


def large_state(n):
    return inputs.vortex_spinor(sweep_like(n, n).grid, n_vortices=10, radius=4.0, seed=70 + n % 7)


def variant_state(nx, ny):
    # a rough state (large seeded phase noise: a broad spectrum in both directions)
    g = variant_problem(nx, ny).grid
    return inputs.gaussian_spinor(g, width=0.5 * min(g.xmax, g.ymax), noise=0.3, seed=nx + 3 * ny, target=TARGET)


def variant_problem(nx, ny):
    # grid spacing 0.025 along the long side, box at least [-0.8, 0.8] along the short one
    return inputs.problem(nx, ny, max(0.8, 0.0125 * nx), max(0.8, 0.0125 * ny), Omega=2.5, delta_slope=0.4,
                          g11=120.0, g22=100.0, g12=110.0, kL=0.8)


def multi_instances():
    prm = inputs.sweep_params(sum(c[2] for c in MULTI), seed=3)
    out, k = [], 0
    for nx, ny, n, xm, ym in MULTI:
        for _ in range(n):
            q = prm[k]
            p = inputs.problem(nx, ny, xm, ym, Omega=q["Omega"], delta_slope=q["delta_slope"], g11=q["g"],
                               g22=q["g"], g12=q["g12"], kL=1.0)
            out.append((p, inputs.vortex_spinor(p.grid, n_vortices=12, radius=4.0, seed=300 + k)))
            k += 1
    return out


def config2_state(i):
    p = inputs.config2(CONFIG2_G12[i])
    return p, inputs.vortex_spinor(p.grid, n_vortices=50, radius=6.0, seed=2 + i)


@pytest.fixture(scope="module")
def refs(orc):
    """Every oracle reference of this module, computed in a spawned pool."""
    jobs, keys = [], []
    for n in LARGE:
        p, psi0 = sweep_like(n, n), large_state(n)
        for mode in MODES:
            jobs.append(oracle_jobs.job_for(p, psi0, LARGE_DTAU, LARGE_STEPS, mode=mode, target=TARGET,
                                            residual=True))
            keys.append(("large", n, mode))
    for nx, ny in VARIANT_GRIDS:
        jobs.append(oracle_jobs.job_for(variant_problem(nx, ny), variant_state(nx, ny), 5e-3, VARIANT_STEPS,
                                        mode=sp.SPGPE_NORM_PER_COMPONENT, target=TARGET))
        keys.append(("variant", nx, ny))
    insts = multi_instances()
    for k in MULTI_SAMPLES:
        p, psi0 = insts[k]
        jobs.append(oracle_jobs.job_for(p, psi0, 5e-3, MULTI_STEPS))
        keys.append(("multi", k))
    for i in range(len(CONFIG2_G12)):
        p, psi0 = config2_state(i)
        jobs.append(oracle_jobs.job_for(p, psi0, 1e-3, CONFIG2_STEPS))
        keys.append(("config2", i))
    return dict(zip(keys, oracle_jobs.run_all(jobs)))


# ------------------------------------------------------------------ cases

@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", LARGE)
def test_large_grid_imaginary_time(refs, n, mode, dtype):
    """512^2 and 1024^2, every coupling on, 60 steps of dtau = 5e-3 from a
    vortex-seeded state: psi, energy, atom numbers and the last-step residual."""
    ref, e_ref, r_ref = refs[("large", n, mode)]
    p = sweep_like(n, n)
    with ctx_for(p, dtype) as c:
        t = to_dev(large_state(n), dtype)
        r = c.step_imag(t, LARGE_DTAU, LARGE_STEPS, mode, TARGET, residual=True)
        got = to_host(t)
        e = c.energy(t)[0]
        nrm = c.norm(t)[0]
    err = np.abs(got - ref).max()
    assert err < tol_psi(dtype, LARGE_STEPS), err
    assert abs(e[0] - e_ref[0]) < tol_energy(dtype) * abs(e_ref[0])
    rt = 1e-12 if dtype == "c128" else 1e-6
    if mode == sp.SPGPE_NORM_PER_COMPONENT:
        assert np.allclose(nrm, TARGET, atol=rt, rtol=0)
    else:
        assert abs(nrm.sum() - sum(TARGET)) < rt
    assert abs(r[0] - r_ref) < (1e-8 * r_ref if dtype == "c128" else 2e-3 + 1e-2 * r_ref)


SCHEDULES = {"plain": {"SPGPE_PERSISTENT": "0"},
             "tma": {"SPGPE_PERSISTENT": "2", "SPGPE_COLPASS": "tma"},
             "warp": {"SPGPE_PERSISTENT": "2", "SPGPE_COLPASS": "warp"}}


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("nx,ny", VARIANT_GRIDS)
def test_pass_variants_imaginary_time(refs, nx, ny, dtype, monkeypatch):
    """Rows and columns of 512 to 2048 points in imaginary time (per-component
    normalisation), each pass variant against the oracle: the plain passes, the
    persistent row pass with the TMA column pass, and (256-row complex64
    grids) the warp-local column pass."""
    ref = refs[("variant", nx, ny)][0]
    p = variant_problem(nx, ny)
    names = ["plain", "tma"] + (["warp"] if dtype == "c64" and ny == 256 else [])
    for name in names:
        monkeypatch.delenv("SPGPE_COLPASS", raising=False)
        for k, v in SCHEDULES[name].items():
            monkeypatch.setenv(k, v)
        with ctx_for(p, dtype) as c:
            t = to_dev(variant_state(nx, ny), dtype)
            c.step_imag(t, 5e-3, VARIANT_STEPS, sp.SPGPE_NORM_PER_COMPONENT, TARGET)
            err = np.abs(to_host(t) - ref).max()
        assert err < (tol_psi(dtype, VARIANT_STEPS) if dtype == "c128" else 2e-5), (name, err)


def test_sweep_batch_size_classes(refs):
    """A multi-size batch of the sweep kind (3 x 256^2, 2 x 512^2, 1 x 1024^2,
    sweep parameters of seed 3, complex64): one sampled instance of each class
    against the oracle after 40 imaginary-time steps."""
    insts = multi_instances()
    with sp.Context.multi(MULTI, "c64") as c:
        for k, (p, _) in enumerate(insts):
            c.set_potentials_separable(k, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
        flat = torch.from_numpy(np.concatenate([x[1].astype(np.complex64).ravel() for x in insts])).cuda()
        c.step_imag(flat, 5e-3, MULTI_STEPS)
        views = c.class_views(flat)
        torch.cuda.synchronize()
        got, k = {}, 0
        for v in views:
            for j in range(v.shape[0]):
                if k in MULTI_SAMPLES:
                    got[k] = v[j].cpu().numpy().astype(np.complex128)
                k += 1
        en = c.energy(flat)
    for k in MULTI_SAMPLES:
        ref, e_ref, _ = refs[("multi", k)]
        assert np.abs(got[k] - ref).max() < 1e-4, k
        assert abs(en[k, 0] - e_ref[0]) < 1e-5 * abs(e_ref[0]), k


@pytest.mark.parametrize("i", range(len(CONFIG2_G12)))
def test_config2_ground_state_problem_first_steps(refs, i):
    """The 1024^2 ground-state problem (box [-24, 24]^2, Omega = 4, delta =
    0.2 y, kL = 2, g11 = g22 = 1000, g12 = 900 / 1000 / 1100, 50 seeded
    vortices): 100 imaginary-time steps in complex64 (FP64 reductions) and in
    complex128 against the oracle."""
    ref, e_ref, _ = refs[("config2", i)]
    p, psi0 = config2_state(i)
    for dtype in ("c64", "c128"):
        with ctx_for(p, dtype) as c:
            t = to_dev(psi0, dtype)
            c.step_imag(t, 1e-3, CONFIG2_STEPS)
            got = to_host(t)
            e = c.energy(t)[0, 0]
        err = np.abs(got - ref).max()
        assert err < tol_psi(dtype, CONFIG2_STEPS), (dtype, err)
        assert abs(e - e_ref[0]) < tol_energy(dtype) * abs(e_ref[0]), dtype
