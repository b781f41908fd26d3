"""The bounded-wait failure path on the GPU, exercised without a fault: a
probe kernel waits (about half a millisecond) on a shared-memory barrier that
nothing completes, gives up, records the timeout in the context's error flags
and exits with nothing in flight.  The host reads SPGPE_ETIMEOUT, the flag is
cleared, and the context keeps stepping correctly."""
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


def _problem():
    return inputs.problem(64, 64, 8.0, 8.0, Omega=1.3, delta_slope=0.2, g11=50.0, g22=45.0, g12=40.0, kL=0.7)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_wait_that_never_completes_reports_timeout_and_the_context_stays_usable(orc, dtype):
    p = _problem()
    g = p.grid
    psi0 = inputs.gaussian_spinor(g, seed=7)
    with sp.Context(g.nx, g.ny, g.xmax, g.ymax, dtype) as c:
        c.set_potentials(p.V, p.delta, p.Omega, p.g11, p.g22, p.g12, p.kL)
        assert c.wait_probe(1 << 20) == sp.SPGPE_ETIMEOUT
        assert "wait limit" in sp.spgpe_last_error(c.handle)
        assert c.wait_probe(0) == sp.SPGPE_ETIMEOUT  # a zero budget gives up at once
        t = torch.from_numpy(psi0.astype(np.complex64 if dtype == "c64" else np.complex128)).cuda()
        c.step_real(t, 1e-3, 10)
        c.sync()  # the flag was cleared: no error left behind
        got = t.cpu().numpy().astype(np.complex128)
    m = orc.Model(g.nx, g.ny, g.xmax, g.ymax, V=p.V, delta=p.delta, Omega=p.Omega,
                  g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    ref = m.step(psi0, 1e-3, 10)
    assert np.abs(got - ref).max() < (1e-5 if dtype == "c64" else 1e-11)


def test_probe_on_a_multi_size_context():
    with sp.Context.multi([(32, 32, 2, 4.0, 4.0), (64, 64, 1, 8.0, 8.0)], "c64") as c:
        assert c.wait_probe(1 << 16) == sp.SPGPE_ETIMEOUT
        assert c.wait_probe(1 << 16) == sp.SPGPE_ETIMEOUT
