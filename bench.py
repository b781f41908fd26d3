"""Benchmark of the fused two-component TSSP step on GB300.

Workload (one "step" = one Strang step S(dt) of Sec. 3.2 over the whole batch):
B independent instances of the 256 x 256 real-time problem (box [-10,10]^2,
harmonic trap, Raman coupling Omega = 2, detuning delta = 0.5 y, kL = 1,
g11 = g22 = g12 = 200, dt = 5e-4, complex64), each started from the ground
state of the 64 x 64 two-component problem (g = 100/100/95) upsampled
spectrally to 256^2 with seeded phase noise per instance.  With B = 256 the
batch is 256 MiB, twice the L2 size, so every timed step streams from HBM
(no L2 flush needed).

Prints one JSON line: grid-point-steps/s (points of one component x steps x
instances, the paper's N of Sec. 5), the roofline of the dominant kernel, the
end-to-end figure through the C ABI with host buffers, the CPU oracle timed on
the host cores, and the SM clocks sampled during the timed region.

``--impl reference`` times the FP64 CPU oracle on the same workload instead
(one instance per step, a bounded sample).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2010_15069_gb300 import inputs  # noqa: E402

NX = NY = 256
DT = 5e-4
DEFAULT_INSTANCES = 256
BYTES_PER_PT_PASS = {"c64": 32, "c128": 64}  # read + write both components, one pass
PASSES_PER_STEP = 2
CUFFT_STEPS = 20
IMAG_STEPS = 100


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ inputs

def ground_state_gpu():
    """Ground state of the 64^2 problem computed by this library (c128)."""
    import torch
    import paper_2010_15069_gb300 as sp
    p = inputs.config0()
    with sp.Context(64, 64, 10.0, 10.0, "c128") as c:
        c.set_potentials(p.V, p.delta, p.Omega, p.g11, p.g22, p.g12, p.kL)
        t = torch.from_numpy(inputs.gaussian_spinor(p.grid, seed=0)).cuda()
        c.step_imag(t, 1e-3, 2000, 1, (0.5, 0.5))
        torch.cuda.synchronize()
        return t.cpu().numpy()


def initial_states(B, ground, first=0):
    """psi0(i): instance first + i of the sweep (its phase noise is seeded by
    that global index, so the ranks of a multi-GPU run step distinct
    instances)."""
    base = inputs.upsample_spectral(ground, NX, NY)

    def psi0(i):
        ph = 1e-3 * (2.0 * inputs.uniform01(1000 + first + i, 2 * NX * NY) - 1.0)
        return base * np.exp(1j * ph.reshape(2, NY, NX))
    return psi0


def instance_range(rank, world, per_rank):
    """(first, count) of the global instances rank `rank` of `world` steps:
    weak scaling, each rank a disjoint slice of per_rank instances and no
    data exchanged between ranks."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return rank * per_rank, per_rank


def max_over_ranks(x, dist=None, device="cpu"):
    """The maximum of a per-rank scalar over all ranks (x itself on one)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(B, dtype="c64", ground=None, stream=None, first=0):
    """(context, device batch tensor, psi0(i)) of the benchmark workload:
    instances first .. first + B - 1."""
    import torch
    import paper_2010_15069_gb300 as sp
    if ground is None:
        ground = ground_state_gpu()
    psi0 = initial_states(B, ground, first)
    p = inputs.config1(NX)
    c = sp.Context(NX, NY, 10.0, 10.0, dtype, ninst=B, stream=stream)
    c.set_potentials_separable(-1, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    npt = np.complex64 if dtype == "c64" else np.complex128
    host = np.empty((B, 2, NY, NX), dtype=npt)
    for i in range(B):
        host[i] = psi0(i)
    t = torch.from_numpy(host).cuda()
    torch.cuda.synchronize()
    return c, t, psi0


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.rows = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is None:
            return
        time.sleep(0.2)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k].lower() == "active"})
        under_load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(under_load) if under_load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------- time to residual

TTR_GRID, TTR_BOX, TTR_DTAU, TTR_TOL, TTR_MAX, TTR_CHECK = 256, 12.0, 5e-3, 1e-8, 60000, 250


def ttr_problems(B):
    """B instances of the parameter sweep (g log-uniform in [50, 2000], g12/g in
    [0.8, 1.2], Omega in [0, 6], detuning gradient in [0, 1], kL = 1, seed 3) on
    256^2 over [-12, 12]^2, each from a vortex-seeded spinor (20 vortices)."""
    n, L = TTR_GRID, TTR_BOX
    prm = inputs.sweep_params(B, seed=3)
    probs = [inputs.problem(n, n, L, L, Omega=q["Omega"], delta_slope=q["delta_slope"], g11=q["g"], g22=q["g"],
                            g12=q["g12"], kL=1.0) for q in prm]
    psi0 = np.stack([inputs.vortex_spinor(probs[0].grid, n_vortices=20, radius=5.0, seed=300 + i)
                     for i in range(B)])
    return probs, psi0


def time_to_residual(B):
    """Wall time until every instance has residual <= 1e-8, has stalled (its
    best residual not halved in 40 checks) or has used its step budget: the
    plain FP64 path (one complex128 context per instance, one after another)
    against the batched complex64 -> complex128 ladder (one context for the
    whole batch, finished instances frozen)."""
    import torch
    import paper_2010_15069_gb300 as sp
    probs, psi0 = ttr_problems(B)
    n, L = TTR_GRID, TTR_BOX

    def ctx(ninst, idx):
        c = sp.Context(n, n, L, L, "c128", ninst)
        for k, i in enumerate(idx):
            p = probs[i]
            c.set_potentials_separable(k, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
        return c

    plain_s, plain_res, plain_steps, plain = 0.0, [], [], []
    for i in range(B):
        with ctx(1, [i]) as c:
            t = torch.from_numpy(psi0[i].copy()).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res, st = c.relax(t, TTR_DTAU, TTR_TOL, TTR_MAX, TTR_CHECK, give_up=True)
            plain_s += time.perf_counter() - t0
            plain_res.append(float(res[0]))
            plain_steps.append(st[1])
            plain.append(t.cpu().numpy())
    with ctx(B, range(B)) as c:
        t = torch.from_numpy(psi0.copy()).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, st = c.relax(t, TTR_DTAU, TTR_TOL, TTR_MAX, TTR_CHECK, ladder=True, give_up=True)
        ladder_s = time.perf_counter() - t0
        e_lad = c.energy(t)[:, 0]
        lad = t.cpu().numpy()
    with ctx(B, range(B)) as c:
        e_pl = c.energy(torch.from_numpy(np.stack(plain)).cuda())[:, 0]
    both = [i for i in range(B) if plain_res[i] <= TTR_TOL and res[i] <= TTR_TOL]
    return {"workload": f"{B} sweep instances, {n}x{n}, box [-{L:g},{L:g}]^2, kL=1, vortex-seeded, "
                        f"dtau={TTR_DTAU:g}, check every {TTR_CHECK} steps, at most {TTR_MAX} steps per stage, "
                        f"instances whose best residual has not halved in 40 checks given up",
            "tol": TTR_TOL, "plain_fp64_unbatched_s": plain_s, "batched_ladder_s": ladder_s,
            "speedup": plain_s / ladder_s,
            "converged": {"plain": sum(r <= TTR_TOL for r in plain_res), "ladder": int((res <= TTR_TOL).sum()),
                          "of": B},
            "steps": {"plain_c128_per_instance": plain_steps, "ladder_c64": st[0], "ladder_c128": st[1]},
            "agreement": {"max_rel_energy_diff": float(np.max(np.abs(e_lad[both] - e_pl[both]) / np.abs(e_pl[both])))
                          if both else None,
                          "max_abs_dpsi": float(np.abs(lad[both] - np.stack(plain)[both]).max()) if both else None}}


# ------------------------------------------------------- uneven sweep batch

SWEEP_CLASSES = [(256, 64), (512, 16), (1024, 4)]   # (grid, instances): 12.58 M points per component
SWEEP_BOX, SWEEP_DTAU = 12.0, 5e-3


def sweep_throughput(steps=40):
    """Imaginary-time steps of the uneven sweep batch (64 x 256^2 + 16 x 512^2 +
    4 x 1024^2, complex64, box [-12, 12]^2, kL = 1, per-instance g, g12, Omega,
    detuning gradient from the sweep generator) as one multi-size batch (size
    classes side by side on their own streams) and as three same-size contexts
    run one after another; grid-point-steps/s of each."""
    import torch
    import paper_2010_15069_gb300 as sp
    total = sum(k for _, k in SWEEP_CLASSES)
    prm = inputs.sweep_params(total, seed=3)
    classes = [(n, n, k, SWEEP_BOX, SWEEP_BOX) for n, k in SWEEP_CLASSES]
    probs, i = [], 0
    for n, k in SWEEP_CLASSES:
        for _ in range(k):
            q = prm[i]
            probs.append(inputs.problem(n, n, SWEEP_BOX, SWEEP_BOX, Omega=q["Omega"], delta_slope=q["delta_slope"],
                                        g11=q["g"], g22=q["g"], g12=q["g12"], kL=1.0))
            i += 1
    psi = [inputs.gaussian_spinor(p.grid, width=3.0, seed=40 + j).astype(np.complex64) for j, p in enumerate(probs)]
    pts = sum(n * n * k for n, k in SWEEP_CLASSES)
    stream = torch.cuda.Stream()

    def timed(run):
        run(3)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run(steps)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e-3

    with sp.Context.multi(classes, "c64", stream=stream) as c:
        for j, p in enumerate(probs):
            c.set_potentials_separable(j, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
        flat = torch.from_numpy(np.concatenate([x.ravel() for x in psi])).cuda()
        c.autotune(flat, 5e-4)
        t_multi = timed(lambda k: c.step_imag(flat, SWEEP_DTAU, k))
    ctxs, bufs, j = [], [], 0
    for n, k in SWEEP_CLASSES:
        cc = sp.Context(n, n, SWEEP_BOX, SWEEP_BOX, "c64", ninst=k, stream=stream)
        for q in range(k):
            p = probs[j + q]
            cc.set_potentials_separable(q, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
        buf = torch.from_numpy(np.stack(psi[j:j + k])).cuda()
        cc.autotune(buf, 5e-4)
        ctxs.append(cc)
        bufs.append(buf)
        j += k
    t_seq = timed(lambda k: [cc.step_imag(b, SWEEP_DTAU, k) for cc, b in zip(ctxs, bufs)])
    for cc in ctxs:
        cc.close()
    return {"workload": "64 x 256^2 + 16 x 512^2 + 4 x 1024^2 instances (12.58 M points per component), c64, "
                        f"imaginary time dtau={SWEEP_DTAU:g}, {steps} steps, sweep parameters (seed 3)",
            "multi_size_batch_pt_steps_per_s": pts * steps / t_multi,
            "same_size_contexts_in_turn_pt_steps_per_s": pts * steps / t_seq,
            "ratio": t_seq / t_multi}


# ------------------------------------------------------- single large instance

SINGLE_SIZES = (2048, 4096)
SINGLE_BOX = 24.0
L2_BYTES = 129e6


def single_instance(steps=200, cufft_steps=40, tune=True):
    """Real time on one large instance: 2048^2 (67 MB of complex64 spinor,
    inside L2) and 4096^2 (268 MB, above it); box [-24, 24]^2, Omega = 2,
    detuning slope 0.2, g11 = g22 = 1000, g12 = 900, kL = 1, dt = 5e-4, the
    trap quenched to omega = 1.1 from a 20-vortex seeded state (seed 4; the
    4096^2 state is the 2048^2 one interpolated spectrally).  The fused passes
    (autotuned unless the schedule is pinned) against the cuFFT comparator on
    the same state (the paper's step structure: cuFFT 2D transforms and
    separate elementwise kernels), with the fused passes' per-kernel times."""
    import torch
    import paper_2010_15069_gb300 as sp
    peak, _ = peaks()
    stream = torch.cuda.Stream()
    seed_state, out = None, []

    def timed(run, k):
        run(3)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run(k)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e-3

    for n in SINGLE_SIZES:
        p = inputs.problem(n, n, SINGLE_BOX, SINGLE_BOX, omega=1.1, Omega=2.0, delta_slope=0.2,
                           g11=1000.0, g22=1000.0, g12=900.0, kL=1.0)
        if seed_state is None:
            seed_state = inputs.vortex_spinor(
                inputs.problem(n, n, SINGLE_BOX, SINGLE_BOX).grid, n_vortices=20, radius=6.0, seed=4)
            psi = seed_state
        else:
            psi = inputs.upsample_spectral(seed_state, n, n)
        with sp.Context(n, n, SINGLE_BOX, SINGLE_BOX, "c64", ninst=1, stream=stream) as c:
            c.set_potentials_separable(-1, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
            t = torch.from_numpy(np.ascontiguousarray(psi.astype(np.complex64))).cuda()
            choice = c.autotune(t, DT)[0] if tune else None
            sec = timed(lambda k: c.step_real(t, DT, k), steps)
            c.set_timing(True)
            c.step_real(t, DT, steps)
            kt = c.timing()
            c.set_timing(False)
            sec_ref = timed(lambda k: c.cufft_step_real(t, DT, k), cufft_steps)
        nbytes = 2 * n * n * 8
        fused = n * n * steps / sec
        ref = n * n * cufft_steps / sec_ref
        out.append({"grid": n, "spinor_mb": nbytes / 1e6, "l2_resident": nbytes < L2_BYTES,
                    "fused_pt_steps_per_s": fused, "ms_per_step": sec / steps * 1e3,
                    "step_frac": 2 * BYTES_PER_PT_PASS["c64"] * n * n * steps / sec / 1e9 / peak,
                    "cufft_comparator_pt_steps_per_s": ref, "fused_over_cufft": fused / ref,
                    "kernel_ms": {k: {"launches": v[0], "avg_ms": v[1] / v[0]} for k, v in kt.items()},
                    "schedule": None if choice is None else
                    {"persistent_row": bool(choice[0] & 1),
                     "column_pass": ["plain", "persistent TMA", "warp-local TMA"][int(choice[0]) >> 1]}})
    return {"workload": "one instance, real time, box [-24,24]^2, Omega=2, delta=0.2y, g=1000, g12=900, kL=1, "
                        "dt=5e-4, trap quenched to omega=1.1, 20-vortex seeded state (seed 4), c64",
            "steps": steps, "cufft_steps": cufft_steps, "sizes": out}


# ------------------------------------------------------- warm-start network

def fno_flops(n, cin=6, cout=4, W=64, M=32, L=4, H=128):
    """Multiply-add count x 2 of one forward pass of the warm-start FNO on n x n
    (the contractions as the kernels run them: the truncated DFTs as products
    with twiddle matrices, complex products counted as 4 real)."""
    P = n * n
    lift = 2 * P * W * cin
    layer = (2 * W * n * n * 2 * M          # along x (real x interleaved complex)
             + 8 * 2 * M * M * n * W         # along y (complex)
             + 8 * W * W * 2 * M * M         # per-mode channel mixing
             + 8 * n * M * 2 * M * W         # inverse along y
             + 2 * W * n * 2 * M * n         # real part of the inverse along x
             + 2 * P * W * W)                # pointwise W_l
    proj = 2 * P * W * H + 2 * P * H * cout
    return lift + L * layer + proj


def fno_throughput(n=256, batch=4, steps=10):
    """Training steps (forward, backward, Adam) of the warm-start FNO at its full
    size (width 64, 32 modes, 4 layers, 67.1 M parameters) on n x n inputs:
    samples/s and the achieved FP32 rate (training = 3 forward passes) against
    the FP32 FMA peak of the CUDA cores at the sampled clock."""
    import torch
    import paper_2010_15069_gb300 as sp
    rng = np.random.default_rng(0)
    a = torch.from_numpy(rng.standard_normal((batch, 6, n, n)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.standard_normal((batch, 4, n, n)).astype(np.float32)).cuda()
    with sp.FNO(6, 4, width=64, modes=32, layers=4, hidden=128, seed=0) as f:
        f.train_step(a, y, 1e-4)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            f.train_step(a, y, 1e-4)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3 / steps
    flop = 3 * fno_flops(n) * batch
    return {"workload": f"FNO width 64, 32 modes, 4 layers, hidden 128 (67.1 M parameters), {n}x{n}, batch {batch}, "
                        "bfloat16 weights, FP32 accumulate, one Adam step per batch",
            "ms_per_train_step": sec * 1e3, "samples_per_s": batch / sec,
            "achieved_tflops": flop / sec / 1e12, "bound": "alu"}


# ------------------------------------------------------------- CPU oracle

def oracle_rate(budget_s=12.0, max_steps=400):
    """The FP64 oracle on one instance of the workload: (pt-steps/s, steps, seconds)."""
    import oracle
    p = inputs.config1(NX)
    m = oracle.Model(NX, NY, 10.0, 10.0, V=p.V, delta=p.delta, Omega=p.Omega,
                     g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    psi = inputs.gaussian_spinor(p.grid, seed=0)
    t0 = time.perf_counter()
    psi = m.step(psi, DT, 1)
    one = time.perf_counter() - t0
    n = int(max(1, min(max_steps, budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    m.step(psi, DT, n)
    dt = time.perf_counter() - t0
    return NX * NY * n / dt, n, dt


def copy_ceiling(t, reps=5):
    """Pinned host <-> device copy rates of one batch-sized buffer, GB/s: in
    alone, out alone, and both directions at once on two streams (the bound
    of an end-to-end step that moves the batch in and out)."""
    import torch
    host_in = torch.empty(tuple(t.shape), dtype=t.dtype, pin_memory=True)
    host_out = torch.empty(tuple(t.shape), dtype=t.dtype, pin_memory=True)
    dev = torch.empty_like(t)
    nbytes = t.numel() * t.element_size()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def h2d():
        with torch.cuda.stream(s_in):
            dev.copy_(host_in, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s_out):
            host_out.copy_(t, non_blocking=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    t_in, t_out = timed(h2d), timed(d2h)
    t_both = timed(lambda: (h2d(), d2h()))
    return {"h2d_gbs": nbytes / t_in / 1e9, "d2h_gbs": nbytes / t_out / 1e9,
            "both_directions_gbs": 2 * nbytes / t_both / 1e9, "bytes": nbytes}


def _oracle_worker(seed, budget_s):
    """One pool worker: oracle steps on its own instance for about budget_s."""
    import oracle
    p = inputs.config1(NX)
    m = oracle.Model(NX, NY, 10.0, 10.0, V=p.V, delta=p.delta, Omega=p.Omega,
                     g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    psi = m.step(inputs.gaussian_spinor(p.grid, seed=seed), DT, 1)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        psi = m.step(psi, DT, 10)
        n += 10
    return NX * NY * n, time.perf_counter() - t0


def oracle_rate_all_cores(budget_s=8.0):
    """The same oracle, one independent instance per host core in a spawned
    process pool (the oracle itself is single-threaded and unchanged):
    (aggregate pt-steps/s, workers, seconds)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_worker, [(i, budget_s) for i in range(cores)])
    wall = time.perf_counter() - t0
    return sum(r[0] / r[1] for r in res), cores, wall


KERNEL_SOURCES = ["fft_core.cuh", "kernels.cuh", "kernels_persist.cuh", "fastmath.cuh", "async_copy.cuh",
                  "internal.h", "launch_row.cuh", "launch_col.cuh"]


def kernel_source_hash():
    """Hash of the code of the kernel sources (line comments, trailing blanks
    and empty lines left out, so that editing a comment keeps the profiles)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2010_15069_gb300", "csrc", f), encoding="utf-8") as fh:
            for ln in fh:
                code = ln.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_traffic(key):
    """DRAM bytes per launch from a committed ncu summary under profiles/, or
    None when no summary covers this kernel or the kernel sources changed since
    the counters were taken (summaries record the hash of the sources)."""
    import glob
    cur = kernel_source_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            lines = f.read().splitlines()
        srcs = [ln.split(":", 1)[1].strip() for ln in lines if ln.startswith("kernel-sources:")]
        if not srcs or srcs[0] != cur:
            continue
        for ln in lines:
            parts = ln.split()
            if len(parts) == 3 and parts[0] == "traffic_bytes_per_launch" and parts[1] == key:
                return int(parts[2])
    return None


def torch_sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ arms

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    p = inputs.config1(NX)
    m = oracle.Model(NX, NY, 10.0, 10.0, V=p.V, delta=p.delta, Omega=p.Omega,
                     g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    psi = inputs.gaussian_spinor(p.grid, seed=0)
    psi = m.step(psi, DT, args.warmup)
    t0 = time.perf_counter()
    m.step(psi, DT, args.steps)
    el = time.perf_counter() - t0
    value = NX * NY * args.steps / el
    line = {
        "impl": "reference", "metric": "grid-point-steps/s", "value": value, "unit": "pt-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.instances, args.dtype),
        "cpu_baseline": {"value": value, "unit": "pt-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"one 256x256 instance of the batch, {args.steps} Strang steps"},
        "e2e": {"value": value, "unit": "pt-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(B, dtype):
    return {"workload": f"256x256 real-time two-component GPE x {B} instances (Omega=2, delta=0.5y, kL=1, "
                        f"g=200, dt=5e-4), {dtype}",
            "grid": [NX, NY], "instances": B, "dt": DT, "box": [-10.0, 10.0],
            "l2": "batch larger than L2 (no flush)" if B * NX * NY * 16 > 129e6 else "L2-resident batch",
            "parallelism": "instances sharded per GPU"}


def run_fused(args):
    import torch
    import paper_2010_15069_gb300 as sp
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B, dtype = args.instances, args.dtype
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        first, _ = instance_range(rank, world, B)
        c, t, _ = make_workload(B, dtype, stream=stream, first=first)
    pts = B * NX * NY
    if args.schedule == "auto":
        # the library's autotuner picks the pass variants for this batch (scratch copy; psi unchanged)
        choice, tune_ms = c.autotune(t, DT)
    else:
        # a fixed schedule (e.g. for a profiler run, under which the tuner's timings mean nothing);
        # set through the environment variable the context reads when it is created
        choice, tune_ms = np.array([{"persistent": 3, "warp": 5, "plain": 0}[args.schedule]]), None

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    c.step_real(t, DT, args.warmup)
    barrier()
    # timed region: K steps in one call (the steady-state cost of a long run)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        start.record(stream)
        c.step_real(t, DT, args.steps)
        stop.record(stream)
        launches = c.last_launches()
        barrier()
    ms = max_over_ranks(start.elapsed_time(stop), dist, "cuda")
    value = world * pts * args.steps / (ms * 1e-3)

    # per-kernel event timing over a second run of the same timed region
    c.set_timing(True)
    c.step_real(t, DT, args.steps)
    kt = c.timing()
    c.set_timing(False)
    kinds = {k: v for k, v in kt.items() if k.startswith(("row_real_fused", "col_real"))}
    dom = max(kinds, key=lambda k: kinds[k][1])
    n_dom, ms_dom = kinds[dom]
    avg_s = ms_dom * 1e-3 / n_dom
    alg_bytes = BYTES_PER_PT_PASS[dtype] * pts
    peak, peak_kind = peaks()
    achieved = alg_bytes / avg_s / 1e9
    traffic = measured_traffic(f"{dom}:{dtype}:{B}")

    # end to end through the C ABI with pinned host buffers: H2D, one step, D2H
    host = torch.empty(tuple(t.shape), dtype=t.dtype, pin_memory=True)
    host.copy_(t)
    hnp = host.numpy()
    c.step_real(hnp, DT, 1)
    e2e_steps = max(3, min(args.steps, 20))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        c.step_real(hnp, DT, 1)
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e_value = world * pts * e2e_steps / e2e_s
    psi_bytes = t.numel() * t.element_size()
    ceiling = copy_ceiling(t)

    # the paper's step structure on the same batch: cuFFT 2D transforms and
    # separate elementwise kernels (a library comparator, not the product path)
    c.cufft_step_real(t, DT, 3)
    barrier()
    start.record(stream)
    c.cufft_step_real(t, DT, CUFFT_STEPS)
    stop.record(stream)
    barrier()
    cufft_value = world * pts * CUFFT_STEPS / (max_over_ranks(start.elapsed_time(stop), dist, "cuda") * 1e-3)

    # imaginary time on the same batch: three passes per step, the
    # renormalisation placed after the whole step (Sec. 3.2)
    c.step_imag(t, DT, 3)
    barrier()
    start.record(stream)
    c.step_imag(t, DT, IMAG_STEPS)
    stop.record(stream)
    barrier()
    imag_s = max_over_ranks(start.elapsed_time(stop), dist, "cuda") * 1e-3
    c.set_timing(True)
    c.step_imag(t, DT, IMAG_STEPS)
    kti = c.timing()
    c.set_timing(False)
    imag = {"value": world * pts * IMAG_STEPS / imag_s, "unit": "pt-steps/s", "steps": IMAG_STEPS, "dtau": DT,
            "ms_per_step": imag_s / IMAG_STEPS * 1e3, "bytes_per_pt_step": 3 * BYTES_PER_PT_PASS[dtype],
            "step_frac": 3 * alg_bytes * IMAG_STEPS / imag_s / 1e9 / peak,
            "kernel_ms": {k: {"launches": v[0], "avg_ms": v[1] / v[0]} for k, v in kti.items()}}
    c.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = cpu_all = None
    if world == 1:
        rate, n, el = oracle_rate()
        cpu = {"value": rate, "unit": "pt-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"one 256x256 instance, {n} FP64 Strang steps in {el:.1f} s (single thread)"}
        rate, cores, el = oracle_rate_all_cores()
        cpu_all = {"value": rate, "unit": "pt-steps/s", "cores": cores, "kind": "oracle",
                   "sample": f"one 256x256 instance per core, FP64 Strang steps for about 8 s each "
                             f"({el:.1f} s wall), spawned process pool"}
    line = {
        "metric": "grid-point-steps/s", "value": value, "unit": "pt-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if dtype == "c64" else "f64", "data": "synthetic",
        "config": dict(workload_config(B, dtype),
                       schedule={"persistent_row": bool(choice[0] & 1),
                                 "column_pass": ["plain", "persistent TMA", "warp-local TMA"][int(choice[0]) >> 1],
                                 "chosen_by": args.schedule,
                                 "autotune_ms_per_step": float(tune_ms[0]) if tune_ms is not None else None}),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_s * 1e3,
                     "peak_source": peak_kind,
                     "step_frac": (PASSES_PER_STEP * alg_bytes * args.steps / (ms * 1e-3) / 1e9) / peak},
        "kernel_ms": {k: {"launches": v[0], "avg_ms": v[1] / v[0]} for k, v in kt.items()},
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "imag_batch": imag,
        "cufft_comparator": {"value": cufft_value, "unit": "pt-steps/s", "steps": CUFFT_STEPS,
                             "what": "same batch and dt, cuFFT 2D C2C transforms + separate R and K kernels "
                                     "(the paper's step structure)",
                             "fused_over_cufft": value / cufft_value},
        "e2e": {"value": e2e_value, "unit": "pt-steps/s", "h2d_bytes_per_step": psi_bytes,
                "d2h_bytes_per_step": psi_bytes, "steps": e2e_steps,
                "copy_gbs": 2 * psi_bytes * e2e_steps / e2e_s / 1e9, "copy_ceiling": ceiling,
                "frac_of_copy_ceiling": 2 * psi_bytes * e2e_steps / e2e_s / 1e9 / ceiling["both_directions_gbs"]},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if world == 1 and args.ttr_instances > 0:
        line["time_to_residual"] = time_to_residual(args.ttr_instances)
    if world == 1 and args.single:
        line["single_instance"] = single_instance(args.single_steps, tune=args.schedule == "auto")
    if world == 1 and args.sweep:
        line["uneven_sweep"] = sweep_throughput()
    if world == 1 and args.fno:
        fn = fno_throughput()
        sm = line["clocks"].get("sm_mhz") or 2070.0
        # FP32 FMA peak of the CUDA cores: SMs x 128 lanes x 2 flop x clock
        peak = torch_sm_count() * 128 * 2 * sm * 1e6 / 1e12
        fn.update(peak_tflops=peak, frac=fn["achieved_tflops"] / peak,
                  peak_source="derived: SMs x 128 FP32 lanes x 2 x sampled SM clock")
        line["warm_start_fno"] = fn
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["fused", "reference"], default="fused")
    ap.add_argument("--instances", type=int, default=DEFAULT_INSTANCES)
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c64")
    ap.add_argument("--schedule", choices=["auto", "persistent", "warp", "plain"], default="auto",
                    help="pass variants: autotuned (default) or fixed")
    ap.add_argument("--sweep", type=int, default=1, help="1: also time the uneven sweep batch (0: skip)")
    ap.add_argument("--single", type=int, default=1,
                    help="1: also time one 2048^2 and one 4096^2 instance against the cuFFT comparator (0: skip)")
    ap.add_argument("--single-steps", type=int, default=200, help="timed steps of each single-instance run")
    ap.add_argument("--fno", type=int, default=1, help="1: also time training of the warm-start FNO (0: skip)")
    ap.add_argument("--ttr-instances", type=int, default=8,
                    help="sweep instances of the time-to-residual comparison (0: skip it)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_2010_15069_gb300 import build
        build.build()
        if args.schedule != "auto":
            os.environ["SPGPE_PERSISTENT"] = "0" if args.schedule == "plain" else "2"
            if args.schedule != "plain":
                os.environ["SPGPE_COLPASS"] = "warp" if args.schedule == "warp" else "tma"
        run_fused(args)


if __name__ == "__main__":
    main()
