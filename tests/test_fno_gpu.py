"""The FNO of the learned warm start (spgpe_fno_*) against the FP64 oracle
(oracle/fno.py), through the C ABI: forward pass, loss and the gradient of
every parameter tensor, one Adam step, and a training run that learns.

The CUDA path multiplies with the weights rounded to bfloat16 and accumulates
in float32; the oracle runs in FP64 on the same rounded weights, so the
comparisons allow float32 accumulation error only.
"""
import numpy as np
import pytest

import paper_2010_15069_gb300 as sp
from oracle import fno as ofno

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2010_15069_gb300 import build
    build.build()
    sp.load()


SMALL = dict(cin=3, cout=4, width=8, modes=4, layers=2, hidden=16)
FULL = dict(cin=6, cout=4, width=64, modes=32, layers=4, hidden=128)   # the warm start's architecture


def setup(cfg, n, B, seed):
    rng = np.random.default_rng(seed)
    sh = ofno.Shapes(cfg["cin"], cfg["cout"], cfg["width"], cfg["modes"], cfg["layers"], cfg["hidden"])
    f = sp.FNO(**cfg, seed=seed)
    theta = f.get_params().astype(np.float64)
    theta += rng.uniform(-0.05, 0.05, theta.size)            # move off the initial biases of zero
    f.set_params(theta.astype(np.float32))
    theta = f.get_params().astype(np.float64)
    a = rng.standard_normal((B, cfg["cin"], n, n)).astype(np.float32)
    t = rng.standard_normal((B, cfg["cout"], n, n)).astype(np.float32)
    return sh, f, theta, a, t


def rel(x, y):
    return float(np.linalg.norm(np.ravel(x - y)) / max(np.linalg.norm(np.ravel(y)), 1e-30))


@pytest.mark.parametrize("cfg,n,B", [(SMALL, 16, 2), (SMALL, 32, 3), (FULL, 64, 2)])
def test_forward_loss_and_gradients_match_oracle(cfg, n, B):
    sh, f, theta, a, t = setup(cfg, n, B, 5)
    with f:
        ad, td = torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda()
        out = f.forward(ad).cpu().numpy()
        loss, g, out2 = f.gradient(ad, td)
    assert np.array_equal(out, out2.cpu().numpy())
    w = ofno.round_bf16(theta)
    ref = ofno.forward(sh, w, a.astype(np.float64))
    assert rel(out, ref) < 2e-5
    lo, go = ofno.loss_and_grad(sh, w, a.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lo) < 1e-5 * lo
    gd, god = sh.unpack(g), sh.unpack(go)
    for name, _ in sh.layout():
        assert rel(gd[name], god[name]) < 2e-4, name


def test_adam_step_matches_the_update_rule():
    sh, f, theta, a, t = setup(SMALL, 16, 2, 9)
    with f:
        ad, td = torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda()
        _, g, _ = f.gradient(ad, td)
        f.train_step(ad, td, 1e-3)
        new = f.get_params().astype(np.float64)
    want, _, _ = ofno.adam_step(theta, g.astype(np.float64), np.zeros_like(theta), np.zeros_like(theta), 1, 1e-3)
    assert np.abs(new - want).max() < 1e-6


def test_training_learns_a_teacher_network():
    """A student FNO fits the outputs of a fixed random teacher of the same shape."""
    cfg, n, B = SMALL, 32, 4
    rng = np.random.default_rng(3)
    a = torch.from_numpy(rng.standard_normal((B, cfg["cin"], n, n)).astype(np.float32)).cuda()
    with sp.FNO(**cfg, seed=11) as teacher, sp.FNO(**cfg, seed=12) as student:
        t = teacher.forward(a)
        losses = [student.train_step(a, t, 3e-3) for _ in range(200)]
    assert losses[-1] < 0.05 * losses[0]


def test_tensor_core_products_agree_with_the_cuda_core_products(monkeypatch):
    """The pointwise channel maps with bfloat16 weights run on the tensor cores
    (tcgen05: the float32 activations split into three bfloat16 terms, float32
    accumulation in tensor memory); SPGPE_FNO_TC=0 keeps them on the CUDA cores.
    At the warm start's architecture on a 128^2 grid (128 tiles of 128 points
    per sample) both give the forward pass and every gradient to float32
    accumulation error."""
    sh, _, theta, a, t = setup(FULL, 128, 2, 13)
    res = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("SPGPE_FNO_TC", mode)
        with sp.FNO(**FULL, seed=13) as f:
            f.set_params(theta.astype(np.float32))
            ad, td = torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda()
            loss, g, out = f.gradient(ad, td)
            res[mode] = (loss, g, out.cpu().numpy())
    assert rel(res["1"][2], res["0"][2]) < 1e-5
    assert abs(res["1"][0] - res["0"][0]) < 1e-5 * res["0"][0]
    g1, g0 = sh.unpack(res["1"][1]), sh.unpack(res["0"][1])
    for name, _ in sh.layout():
        assert rel(g1[name], g0[name]) < 1e-4, name
