"""Host-side legs of bench.py that need no GPU: the reference arm (the FP64
oracle timed on the host cores) and the spawned all-cores oracle pool."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line(orc):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "3"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "grid-point-steps/s" and d["unit"] == "pt-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 3 and d["warmup"] == 3
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]


def test_reference_arm_rejects_short_warmup():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "2"], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode != 0 and "warmup" in r.stderr


def test_oracle_pool_uses_every_core(orc):
    import bench
    rate, cores, wall = bench.oracle_rate_all_cores(budget_s=0.3)
    expect = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    assert cores == expect
    assert rate > 0 and wall > 0.3


def test_ground_state_verdict():
    """Two relaxed states of one problem 'match' when both are converged and
    agree up to the global phase, are 'degenerate' when only their energies
    agree (different metastable states), and a 'mismatch' otherwise."""
    import numpy as np
    import bench
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, 8, 8)) + 1j * rng.standard_normal((2, 8, 8))
    b = a * np.exp(0.7j)  # the same state, another global phase
    assert bench.ground_state_verdict(a, b, 1.0, 1.0, 1e-9, 1e-9, 1e-8)[0] == "match"
    c = a + 1e-3 * rng.standard_normal(a.shape)
    assert bench.ground_state_verdict(a, c, 1.0, 1.0 + 1e-7, 1e-9, 1e-9, 1e-8)[0] == "degenerate"
    assert bench.ground_state_verdict(a, b, 1.0, 1.0, 1e-9, 1e-6, 1e-8)[0] == "degenerate"  # b not converged
    assert bench.ground_state_verdict(a, c, 1.0, 1.01, 1e-9, 1e-9, 1e-8)[0] == "mismatch"
