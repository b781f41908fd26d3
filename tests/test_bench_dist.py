"""The multi-GPU host logic of bench.py on CPU: world size 2 over gloo.

Ranks step disjoint slices of the instance sweep (weak scaling, no data
exchanged), the timed region's duration is the maximum over ranks, and under
torchrun the reference arm prints one line from rank 0 while the other rank
exits without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        first, count = bench.instance_range(rank, world, 5)
        slowest = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        seeds = [1000 + first + i for i in range(count)]
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out.put((rank, first, count, slowest, gathered))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_the_sweep_and_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, f0, c0, m0, g0), (r1, f1, c1, m1, g1) = res
    assert (f0, c0, f1, c1) == (0, 5, 5, 5)
    assert m0 == m1 == 2.5  # the slower rank's time, on every rank
    seeds = g0[0] + g0[1]
    assert g0 == g1 and len(set(seeds)) == 10  # disjoint instances, every one stepped once


def test_instance_range_rejects_a_rank_outside_the_world():
    sys.path.insert(0, ROOT)
    import bench
    with pytest.raises(ValueError):
        bench.instance_range(2, 2, 4)
    assert bench.max_over_ranks(3.0) == 3.0


def test_reference_arm_under_torchrun_prints_once(orc):
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
