"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Every case feeds the same seeded inputs (paper_2010_15069_gb300.inputs) to
both sides.  Tolerances: complex128 within 1e-11 max|dpsi| per 100 steps
(different FFT algorithms round differently); complex64 within 1e-4 max|dpsi|
and 1e-5 relative energy after 1000 steps, with the spinor normalised to one
atom (max|psi| ~ 0.56).
"""
import math

import numpy as np
import pytest

import paper_2010_15069_gb300 as sp
from paper_2010_15069_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU only with -m gpu
    pytest.skip("CUDA not available", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2010_15069_gb300 import build
    build.build()
    sp.load()


NPT = {"c64": np.complex64, "c128": np.complex128}


def to_dev(psi, dtype):
    return torch.from_numpy(np.ascontiguousarray(psi.astype(NPT[dtype]))).cuda()


def to_host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def c128_tol(nsteps):
    return 1e-11 * max(1.0, nsteps / 100.0)


def ctx_for(p, dtype, separable=False, ninst=1):
    g = p.grid
    c = sp.Context(g.nx, g.ny, g.xmax, g.ymax, dtype, ninst)
    if separable:
        c.set_potentials_separable(-1, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    else:
        c.set_potentials(p.V, p.delta, p.Omega, p.g11, p.g22, p.g12, p.kL)
    return c


def model_for(orc, p):
    g = p.grid
    return orc.Model(g.nx, g.ny, g.xmax, g.ymax, V=p.V, delta=p.delta, Omega=p.Omega,
                     g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)


def coupled(nx, ny, g=60.0):
    """All terms on: trap, detuning gradient, uniform Raman, SOC, unequal couplings.
    Grid spacing 0.25 in both directions (box at least [-2, 2])."""
    return inputs.problem(nx, ny, max(2.0, 0.125 * nx), max(2.0, 0.125 * ny), Omega=1.7, delta_slope=0.3,
                          g11=g, g22=0.8 * g, g12=0.9 * g, kL=0.9)


@pytest.fixture(scope="module")
def ground0(orc):
    """Ground state of the 64^2 two-component problem (imaginary time, oracle)."""
    p = inputs.config0()
    m = model_for(orc, p)
    psi0 = inputs.gaussian_spinor(p.grid, seed=0)
    return m.step(psi0, 1e-3, 2000, imag=True, norm_mode=1, target=(0.5, 0.5))


# ------------------------------------------------------------ real time

@pytest.mark.parametrize("nx,ny", [(64, 64), (16, 128), (256, 32), (8, 8), (128, 64), (1024, 16), (4096, 16),
                                   (16, 1024), (16, 4096)])
@pytest.mark.parametrize("separable", [False, True])
def test_real_time_c128_matches_oracle(orc, nx, ny, separable):
    p = coupled(nx, ny)
    psi0 = inputs.gaussian_spinor(p.grid, width=1.2, seed=nx + ny, target=(0.6, 0.4))
    n = 60
    ref = model_for(orc, p).step(psi0, 2e-3, n)
    with ctx_for(p, "c128", separable) as c:
        t = to_dev(psi0, "c128")
        c.step_real(t, 2e-3, n)
        assert c.last_launches() == 2 * n + 1
        got = to_host(t)
    assert np.abs(got - ref).max() < c128_tol(n)


def test_config1_c64_and_c128_side_by_side(orc, ground0):
    """256^2, Omega = 2, delta = 0.5 y, kL = 1, g = 200, dt = 5e-4, from the
    upsampled 64^2 ground state; 1000 steps (bars: c64 1e-4 / 1e-5, c128 1e-10)."""
    p = inputs.config1()
    psi0 = inputs.upsample_spectral(ground0, 256, 256)
    n = 1000
    m = model_for(orc, p)
    ref = m.step(psi0, 5e-4, n)
    e_ref = m.energy(ref)[0]
    for dtype, tol in (("c64", 1e-4), ("c128", c128_tol(n))):
        with ctx_for(p, dtype, separable=True) as c:
            t = to_dev(psi0, dtype)
            c.step_real(t, 5e-4, n)
            got = to_host(t)
            e = c.energy(t)[0, 0]
        assert np.abs(got - ref).max() < tol, dtype
        assert abs(e - e_ref) / abs(e_ref) < (1e-5 if dtype == "c64" else 1e-12), dtype


# ------------------------------------------------------- imaginary time

def test_config0_c128_full_protocol(orc, ground0):
    """64^2, g = 100/100/95: 2000 imaginary steps (per component), then 500 real."""
    p = inputs.config0()
    m = model_for(orc, p)
    psi0 = inputs.gaussian_spinor(p.grid, seed=0)
    with ctx_for(p, "c128") as c:
        t = to_dev(psi0, "c128")
        c.step_imag(t, 1e-3, 2000, sp.SPGPE_NORM_PER_COMPONENT, (0.5, 0.5))
        assert c.last_launches() == 3 * 2000 + 1
        assert np.abs(to_host(t) - ground0).max() < c128_tol(2000)
        c.step_real(t, 1e-3, 500)
        got = to_host(t)
    ref = m.step(ground0, 1e-3, 500)
    assert np.abs(got - ref).max() < c128_tol(2500)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("mode", [sp.SPGPE_NORM_TOTAL, sp.SPGPE_NORM_PER_COMPONENT])
def test_imag_time_with_coupling_and_residual(orc, dtype, mode):
    p = coupled(64, 32)
    psi0 = inputs.vortex_spinor(p.grid, n_vortices=6, radius=3.0, seed=3)
    n = 150
    ref, r_ref = model_for(orc, p).step(psi0, 1e-2, n, imag=True, norm_mode=mode, target=(0.7, 0.3),
                                        residual=True)
    with ctx_for(p, dtype) as c:
        t = to_dev(psi0, dtype)
        r = c.step_imag(t, 1e-2, n, mode, (0.7, 0.3), residual=True)
        got = to_host(t)
        nrm = c.norm(t)[0]
    tol = c128_tol(n) if dtype == "c128" else 2e-5
    assert np.abs(got - ref).max() < tol
    assert abs(r[0] - r_ref) < (1e-8 * r_ref if dtype == "c128" else 2e-3 + 1e-2 * r_ref)
    if mode == sp.SPGPE_NORM_PER_COMPONENT:
        assert np.allclose(nrm, [0.7, 0.3], atol=1e-12 if dtype == "c128" else 1e-6)
    else:
        assert abs(nrm.sum() - 1.0) < (1e-12 if dtype == "c128" else 1e-6)


def test_batch_of_instances_matches_individual_oracle_runs(orc):
    g = inputs.Grid(64, 32, 10.0, 6.0)
    params = inputs.sweep_params(3, seed=3)
    ps = [inputs.problem(64, 32, 10.0, 6.0, Omega=q["Omega"], delta_slope=q["delta_slope"],
                         g11=q["g"], g22=q["g"], g12=q["g12"], kL=0.5 + 0.25 * i)
          for i, q in enumerate(params)]
    psi0 = np.stack([inputs.gaussian_spinor(g, seed=40 + i) for i in range(3)])
    with sp.Context(64, 32, 10.0, 6.0, "c128", ninst=3) as c:
        for i, p in enumerate(ps):
            c.set_potentials_separable(i, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
        t = to_dev(psi0, "c128")
        c.step_imag(t, 5e-3, 40, sp.SPGPE_NORM_TOTAL, (0.5, 0.5))
        c.step_real(t, 1e-3, 40)
        got = to_host(t)
        en = c.energy(t)
    for i, p in enumerate(ps):
        m = model_for(orc, p)
        ref = m.step(m.step(psi0[i], 5e-3, 40, imag=True, norm_mode=0), 1e-3, 40)
        assert np.abs(got[i] - ref).max() < c128_tol(80), i
        assert np.allclose(en[i], m.energy(ref), rtol=1e-11, atol=1e-12), i


# ----------------------------------------------------- energy and norm

@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("separable", [False, True])
def test_energy_and_norm_match_oracle(orc, dtype, separable):
    p = coupled(128, 64)
    psi = inputs.vortex_spinor(p.grid, n_vortices=9, radius=3.0, seed=5, target=(0.55, 0.45))
    m = model_for(orc, p)
    e_ref, n_ref = m.energy(psi), m.norm(psi)
    with ctx_for(p, dtype, separable) as c:
        t = to_dev(psi, dtype)
        e, n = c.energy(t)[0], c.norm(t)[0]
        e_host = c.energy(psi.astype(NPT[dtype]))[0]
    rt = 1e-12 if dtype == "c128" else 2e-6
    assert np.allclose(n, n_ref, rtol=rt, atol=0)
    assert np.allclose(e, e_ref, rtol=rt, atol=rt * abs(e_ref[0]))
    assert np.array_equal(e, e_host)


# ------------------------------------------- paths, splits, comparator

@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_host_spinor_path_is_bit_identical(dtype):
    p = coupled(128, 128)
    psi0 = inputs.gaussian_spinor(p.grid, seed=7).astype(NPT[dtype])
    with ctx_for(p, dtype) as c:
        t = to_dev(psi0, dtype)
        c.step_real(t, 1e-3, 25)
        h = psi0.copy()
        c.step_real(h, 1e-3, 25)
        assert np.array_equal(to_host(t), h.astype(np.complex128))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_host_batch_goes_through_in_chunks_with_the_same_bits(dtype):
    """A host spinor batch is copied in, stepped and copied out in chunks of
    instances (uneven: 11 instances in 8 chunks) with the copies overlapping
    the steps; the result equals stepping the batch on the device."""
    p = coupled(64, 256)
    psi0 = np.stack([inputs.gaussian_spinor(p.grid, seed=60 + i) for i in range(11)]).astype(NPT[dtype])
    with ctx_for(p, dtype, ninst=11) as c:
        t = to_dev(psi0, dtype)
        c.step_real(t, 1e-3, 9)
        c.step_imag(t, 1e-3, 4, sp.SPGPE_NORM_PER_COMPONENT)
        h = psi0.copy()
        c.step_real(h, 1e-3, 9)
        c.step_imag(h, 1e-3, 4, sp.SPGPE_NORM_PER_COMPONENT)
        assert np.array_equal(to_host(t), h.astype(np.complex128))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_split_runs_agree(dtype):
    """Real time: within a call the closing X(dt/4) of one step and the opening
    X(dt/4) of the next are applied as one rotation by the doubled angle; at a
    call boundary they are applied one after the other, so a split run agrees
    to rounding.  Imaginary time has no such merge: bit-identical."""
    p = coupled(64, 128)
    psi0 = inputs.gaussian_spinor(p.grid, seed=8)
    with ctx_for(p, dtype) as c:
        a, b = to_dev(psi0, dtype), to_dev(psi0, dtype)
        c.step_real(a, 1e-3, 30)
        c.step_real(b, 1e-3, 13)
        c.step_real(b, 1e-3, 17)
        tol = 1e-13 if dtype == "c128" else 2e-6
        assert np.abs(to_host(a) - to_host(b)).max() < tol * np.abs(to_host(a)).max()
        b.copy_(a)
        c.step_imag(a, 1e-3, 30, sp.SPGPE_NORM_TOTAL)
        c.step_imag(b, 1e-3, 11)
        c.step_imag(b, 1e-3, 19)
        assert torch.equal(a, b)


@pytest.mark.parametrize("dtype,nx,ny,ninst", [("c64", 8, 8, 2), ("c64", 64, 32, 3), ("c64", 256, 64, 2),
                                               ("c64", 512, 16, 1), ("c64", 2048, 8, 1), ("c64", 4096, 8, 1),
                                               ("c128", 128, 32, 2), ("c128", 512, 16, 1)])
def test_persistent_and_plain_row_passes_agree(dtype, nx, ny, ninst, monkeypatch):
    """The persistent row pass (per-unit prefetch) against the plain one-tile-per-
    block pass: real time bit for bit (same arithmetic), imaginary time to the
    rounding of the FP64 atom-number sums (their grouping differs)."""
    p = coupled(nx, ny)
    psi0 = np.stack([inputs.gaussian_spinor(p.grid, seed=20 + i) for i in range(ninst)])
    out = {}
    for mode in ("0", "2"):
        monkeypatch.setenv("SPGPE_PERSISTENT", mode)
        with ctx_for(p, dtype, ninst=ninst) as c:
            a = to_dev(psi0, dtype)
            c.step_real(a, 1e-3, 7)
            b = a.clone()
            c.step_imag(b, 1e-3, 9, sp.SPGPE_NORM_PER_COMPONENT)
            out[mode] = (to_host(a), to_host(b))
    assert np.array_equal(out["0"][0], out["2"][0])
    tol = 1e-12 if dtype == "c128" else 2e-6
    assert np.abs(out["0"][1] - out["2"][1]).max() < tol


@pytest.mark.parametrize("nx,ninst", [(16, 3), (64, 2), (256, 2), (512, 1)])
def test_column_pass_variants_agree(nx, ninst, monkeypatch):
    """The column pass as one tile per block, as the persistent TMA pass and as
    the warp-local TMA pass (128-byte swizzle, ny = 256, complex64): same
    arithmetic, so the same bits in real time, and in imaginary time between
    the two TMA passes (both beside the persistent row pass; the plain row
    pass groups the FP64 atom-number sums differently)."""
    p = coupled(nx, 256)
    psi0 = np.stack([inputs.gaussian_spinor(p.grid, seed=30 + i) for i in range(ninst)])
    out = {}
    for name, env in (("plain", {"SPGPE_PERSISTENT": "0"}), ("tma", {"SPGPE_PERSISTENT": "2", "SPGPE_COLPASS": "tma"}),
                      ("warp", {"SPGPE_PERSISTENT": "2", "SPGPE_COLPASS": "warp"})):
        monkeypatch.delenv("SPGPE_COLPASS", raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        with ctx_for(p, "c64", ninst=ninst) as c:
            a = to_dev(psi0, "c64")
            c.step_real(a, 1e-3, 6)
            b = a.clone()
            c.step_imag(b, 1e-3, 5, sp.SPGPE_NORM_TOTAL)
            out[name] = (to_host(a), to_host(b))
    for name in ("tma", "warp"):
        assert np.array_equal(out[name][0], out["plain"][0]), name
    assert np.array_equal(out["warp"][1], out["tma"][1])
    assert np.abs(out["tma"][1] - out["plain"][1]).max() < 2e-6


@pytest.mark.parametrize("dtype,ny", [("c64", 1024), ("c64", 2048), ("c64", 4096), ("c128", 1024), ("c128", 2048),
                                      ("c128", 4096)])
def test_tall_columns_against_oracle_and_plain_pass(orc, dtype, ny, monkeypatch):
    """Columns of 1024 to 4096 rows (the persistent TMA column pass with a few
    columns per tile and one 256-row box per 256 rows, and factored stage
    twiddles from a span of 256 on; 16 x ny, two instances):
    real time against the oracle, and bit for bit against the plain pass."""
    p = coupled(16, ny)
    psi0 = np.stack([inputs.gaussian_spinor(p.grid, seed=50 + i) for i in range(2)])
    out = {}
    for mode in ("0", "2"):
        monkeypatch.setenv("SPGPE_PERSISTENT", mode)
        with ctx_for(p, dtype, ninst=2) as c:
            a = to_dev(psi0, dtype)
            c.step_real(a, 1e-3, 4)
            out[mode] = to_host(a)
    assert np.array_equal(out["0"], out["2"])
    m = model_for(orc, p)
    tol = c128_tol(4) if dtype == "c128" else 1e-5
    for i in range(2):
        assert np.abs(out["2"][i] - m.step(psi0[i], 1e-3, 4)).max() < tol


def test_cufft_comparator_matches_oracle(orc):
    p = coupled(64, 64)
    psi0 = inputs.gaussian_spinor(p.grid, seed=9)
    ref = model_for(orc, p).step(psi0, 2e-3, 50)
    with ctx_for(p, "c128") as c:
        t = to_dev(psi0, "c128")
        c.cufft_step_real(t, 2e-3, 50)
        assert np.abs(to_host(t) - ref).max() < c128_tol(50)


# ----------------------------------------------------------- errors

def test_error_statuses():
    g = inputs.Grid(32, 32, 5.0, 5.0)
    with sp.Context(32, 32, 5.0, 5.0, "c64") as c:
        t = to_dev(inputs.gaussian_spinor(g), "c64")
        with pytest.raises(sp.SpgpeError, match="ESTATE"):
            c.step_real(t, 1e-3, 1)
        c.set_potentials(inputs.harmonic(g), g11=1.0)
        with pytest.raises(sp.SpgpeError, match="EINVAL"):
            c.step_real(t, float("nan"), 1)
        with pytest.raises(sp.SpgpeError, match="EINVAL"):
            c.set_potentials(np.full((32, 32), np.inf))
        for bad in (2, 3, 6, 7):  # a normalisation mode other than TOTAL / PER_COMPONENT (| LAGGED)
            with pytest.raises(sp.SpgpeError, match="EINVAL"):
                c.step_imag(t, 1e-3, 1, norm_mode=bad)
        z = torch.zeros_like(t)
        with pytest.raises(sp.SpgpeError, match="ENONFINITE"):
            c.step_imag(z, 1e-3, 3, sp.SPGPE_NORM_TOTAL, residual=True)
        c.step_imag(z, 1e-3, 2)            # asynchronous: reported by the next sync
        with pytest.raises(sp.SpgpeError, match="ENONFINITE"):
            c.sync()
        c.sync()                           # flag cleared
        c.step_real(t, 1e-3, 0)


# ------------------------------------------------ full-size workloads

def test_bench_workload_sampled_instances(orc, ground0):
    """The benchmark's batch (256 instances of the 256^2 real-time problem, c64)
    in its launch configuration; sampled instances against the oracle."""
    import bench
    B, n = 256, 20
    c, t, psi0 = bench.make_workload(B, "c64")
    try:
        norm0 = c.norm(t).sum(axis=1)
        c.step_real(t, bench.DT, n)
        got = t[[0, B // 2, B - 1]].cpu().numpy().astype(np.complex128)
        norm1 = c.norm(t).sum(axis=1)
    finally:
        c.close()
    assert np.allclose(norm1, norm0, rtol=2e-5, atol=0)
    m = model_for(orc, inputs.config1())
    for k, i in enumerate((0, B // 2, B - 1)):
        ref = m.step(psi0(i), bench.DT, n)
        assert np.abs(got[k] - ref).max() < 1e-4, i


def test_largest_grid_2048_c64_error_growth(orc):
    """2048^2 real time (config 4's grid: box [-24,24]^2, dt = 5e-4, trap
    quenched to omega = 1.1, Raman coupling, detuning gradient, SOC, g = 1000,
    g12 = 900) from a 20-vortex seeded state: complex64 against the oracle
    after 50, 100, 150 and 200 steps (the error growth of complex64 at this
    size; bar 1e-4 per the complex64 tolerance)."""
    p = inputs.problem(2048, 2048, 24.0, 24.0, omega=1.1, Omega=2.0, delta_slope=0.2, g11=1000.0, g22=1000.0,
                       g12=900.0, kL=1.0)
    psi = inputs.vortex_spinor(p.grid, n_vortices=20, radius=6.0, seed=4)
    m = model_for(orc, p)
    errs = []
    with ctx_for(p, "c64", separable=True) as c:
        t = to_dev(psi, "c64")
        ref = psi
        for _ in range(4):
            c.step_real(t, 5e-4, 50)
            ref = m.step(ref, 5e-4, 50)
            errs.append(float(np.abs(to_host(t) - ref).max()))
    print("2048^2 complex64 max|dpsi| after 50/100/150/200 steps:", errs)
    assert all(e < 1e-4 for e in errs), errs


def test_largest_grid_2048_c64(orc):
    """2048^2 real time (box [-24,24]^2, dt = 5e-4): three steps against the oracle."""
    p = inputs.problem(2048, 2048, 24.0, 24.0, Omega=2.0, delta_slope=0.2, g11=1000.0, g22=1000.0,
                       g12=900.0, kL=1.0)
    psi0 = inputs.vortex_spinor(p.grid, n_vortices=20, radius=6.0, seed=4)
    ref = model_for(orc, p).step(psi0, 5e-4, 3)
    with ctx_for(p, "c64", separable=True) as c:
        t = to_dev(psi0, "c64")
        c.step_real(t, 5e-4, 3)
        got = to_host(t)
    assert np.abs(got - ref).max() < 1e-5
