"""Benchmark of the fused TSSP passes on GB300.

Headline workload (one "step" = one imaginary-time step of Sec. 3.2, S(dtau)
and the renormalisation, over the whole batch): the parameter-sweep batch of
64 instances at 256^2, 16 at 512^2 and 4 at 1024^2 (12.58 M grid points per
component, 201 MB of complex64 spinor: above the L2 size, so every step
streams from HBM and no flush is needed), box [-12, 12]^2, harmonic trap,
kL = 1, per-instance g (log-uniform in [50, 2000]), g12 / g (in [0.8, 1.2]),
Omega (in [0, 6]) and detuning gradient (in [0, 1]) from the sweep generator
(seed 3), vortex-seeded spinors (20 vortices), dtau = 5e-3, complex64
operators with FP64 reductions and the lagged renormalisation (two passes
over psi per step), run as one multi-size batch whose size classes share the
GPU.  The K timed steps run in one call.

Prints one JSON line: grid-point-steps/s (points of one component x steps x
instances, the paper's N of Sec. 5), the roofline of the dominant kernel, the
same workload with the exact renormalisation and in complex128, the
end-to-end figure through the C ABI with host buffers, the CPU oracle timed on
the host cores, the GPU's measured ceilings and the SM clocks sampled during
the timed region; further objects cover the real-time batch of the 256^2
problem, the cuFFT comparator, time to residual 1e-8, single large instances
and the warm-start network.

``--impl reference`` times the FP64 CPU oracle on the same workload instead
(one 256^2 instance of the sweep per step, a bounded sample).
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

# real-time batch of the 256^2 problem (Omega = 2, delta = 0.5 y, kL = 1, g = 200)
NX = NY = 256
DT = 5e-4
DEFAULT_INSTANCES = 256
BYTES_PER_PT_PASS = {"c64": 32, "c128": 64}  # read + write both components, one pass
PASSES_PER_STEP = 2
CUFFT_STEPS = 20

# imaginary-time sweep batch (the headline)
SWEEP_CLASSES = [(256, 64), (512, 16), (1024, 4)]   # (grid, instances): 12.58 M points per component
SWEEP_BOX, SWEEP_DTAU, SWEEP_KL = 12.0, 5e-3, 1.0
C128_STEPS = 40
TIMING_STEPS = 200


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


# ------------------------------------------------------- sweep batch

def sweep_problems(classes=SWEEP_CLASSES, first=0):
    """(multi-size classes, problems, initial spinors) of the sweep batch: the
    instances with global indices first .. first + total - 1 (parameters from
    the sweep generator, seed 3, drawn in that order; spinors with 20 vortices
    seeded by the global index), grouped by grid size."""
    total = sum(k for _, k in classes)
    prm = inputs.sweep_params(first + total, seed=3)[first:]
    out, probs, psi, i = [], [], [], 0
    for n, k in classes:
        out.append((n, n, k, SWEEP_BOX, SWEEP_BOX))
        for _ in range(k):
            q = prm[i]
            p = inputs.problem(n, n, SWEEP_BOX, SWEEP_BOX, Omega=q["Omega"], delta_slope=q["delta_slope"],
                               g11=q["g"], g22=q["g"], g12=q["g12"], kL=SWEEP_KL)
            probs.append(p)
            psi.append(inputs.vortex_spinor(p.grid, n_vortices=20, radius=5.0, seed=300 + first + i))
            i += 1
    return out, probs, psi


def make_multi(classes, probs, psi, dtype, stream=None):
    """A multi-size context with every instance's potentials, and the batch
    as one flat device tensor."""
    import torch
    import paper_2010_15069_gb300 as sp
    c = sp.Context.multi(classes, dtype, stream=stream)
    for j, p in enumerate(probs):
        c.set_potentials_separable(j, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    npt = np.complex64 if dtype == "c64" else np.complex128
    flat = torch.from_numpy(np.concatenate([x.astype(npt).ravel() for x in psi])).cuda()
    torch.cuda.synchronize()
    return c, flat


def timed_events(stream, run):
    """Seconds of run() between CUDA events on `stream`, synchronised on both sides."""
    import torch
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    run()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) * 1e-3


def kernel_times_in_turn(c, flat, classes, probs, dtype, stream, steps, lagged):
    """Per-kernel CUDA-event times of `steps` imaginary-time steps of each size
    class alone on the GPU (a same-size context over the class's part of the
    batch, the classes one after another on one stream; in the multi-size run
    the classes' kernels overlap, so a kernel's event-bracketed time there would
    include the other classes' work).  [(grid, instances, {kind: (launches, ms)})]."""
    import paper_2010_15069_gb300 as sp
    out, j = [], 0
    for (n, _, k, xm, ym), view in zip(classes, c.class_views(flat)):
        with sp.Context(n, n, xm, ym, dtype, ninst=k, stream=stream) as cc:
            for q in range(k):
                p = probs[j + q]
                cc.set_potentials_separable(q, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
            cc.autotune(view, 5e-4)
            cc.step_imag(view, SWEEP_DTAU, 3, lagged=lagged)
            cc.set_timing(True)
            cc.step_imag(view, SWEEP_DTAU, steps, lagged=lagged)
            out.append((n, k, cc.timing()))
            cc.set_timing(False)
        j += k
    return out


def dominant(per_class):
    """(grid, instances, kind, launches, total ms) of the kernel kind with the
    largest total time among the step's passes."""
    best = None
    for n, k, kt in per_class:
        for kind, (cnt, ms) in kt.items():
            if kind in ("row_imag_open", "row_imag_rescale"):
                continue  # once per call, not part of the steady state
            if best is None or ms > best[4]:
                best = (n, k, kind, cnt, ms)
    return best


# Algorithmic FP64 flops per grid point (both components) of one pass: each
# complex transform of length n counts 5 n log2 n (the usual radix-2 count),
# a row pass runs the inverse and forward x-transforms of both components
# and the two R(dtau/2) halves (48 flops of pointwise operators), a column
# pass the forward and inverse y-transforms and K (12 flops).
def flops_per_point(kind, n):
    lg = math.log2(n)
    if kind.startswith("col"):
        return 2 * 2 * 5 * lg + 12
    return 2 * 2 * 5 * lg + 48


def ceilings():
    import paper_2010_15069_gb300 as sp
    try:
        return sp.spgpe_probe_ceilings()
    except Exception as e:  # measured ceilings are context; the bench goes on without them
        return {"error": str(e)}


def l2_capacity_mib(ceil):
    """Largest probed working set whose read bandwidth is still well above the
    largest set's (HBM) bandwidth: the L2 capacity to within the probe's steps."""
    tab = ceil.get("read_gbs_by_working_set_mib") if isinstance(ceil, dict) else None
    if not tab:
        return None
    hbm = tab[max(tab)]
    inside = [m for m, v in tab.items() if v > 1.5 * hbm]
    return max(inside) if inside else None


# ------------------------------------------------------- time to residual

TTR_CLASSES = [(256, 8), (512, 2), (1024, 1)]   # one eighth of the sweep batch
TTR_TOL, TTR_MAX, TTR_CHECK = 1e-8, 60000, 250


def oracle_fixed_point_residual(p, psi, dtau):
    """The FP64 oracle's discrete-map residual of one exact step from psi: how
    far psi is from the oracle's own fixed point."""
    import oracle
    g = p.grid
    m = oracle.Model(g.nx, g.ny, g.xmax, g.ymax, V=p.V, delta=p.delta, Omega=p.Omega,
                     g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    _, r = m.step(psi, dtau, 1, imag=True, residual=True)
    return r


WS_TRAIN, WS_ITERS, WS_BATCH, WS_LR, WS_SEED = 256, 1200, 4, 1e-3, 33


def train_warm_start():
    """The learned warm start (width 64, 32 modes, 4 Fourier layers, hidden
    128): WS_TRAIN ground states of the sweep generator at 256^2 (parameters
    from seed 33, disjoint from the timed instances' seed 3), relaxed by the
    batched complex64 path with the lagged renormalisation to residual 2e-3 or
    a stall from 20-vortex seeded spinors (the seeding the timed arms use),
    then WS_ITERS Adam steps on random batches of WS_BATCH.  Everything runs
    on the default stream, in order with the tensors it reads.  Returns
    (model, {seconds and losses})."""
    import torch
    import paper_2010_15069_gb300 as sp
    from paper_2010_15069_gb300 import warmstart
    n, L = 256, SWEEP_BOX
    prm = inputs.sweep_params(WS_TRAIN, seed=WS_SEED)
    grid = inputs.Grid(n, n, L, L)
    info = {}
    t0 = time.perf_counter()
    with sp.Context(n, n, L, L, "c64", ninst=WS_TRAIN) as c:
        for i, q in enumerate(prm):
            p = inputs.problem(n, n, L, L, Omega=q["Omega"], delta_slope=q["delta_slope"], g11=q["g"], g22=q["g"],
                               g12=q["g12"], kL=SWEEP_KL)
            c.set_potentials_separable(i, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
        t = torch.from_numpy(np.stack([inputs.vortex_spinor(grid, n_vortices=20, radius=5.0, seed=5000 + i)
                                       for i in range(WS_TRAIN)]).astype(np.complex64)).cuda()
        c.relax(t, SWEEP_DTAU, 2e-3, 20000, TTR_CHECK, give_up=True, lagged=True)
        gs = t.cpu().numpy().astype(np.complex128)
    info["ground_states_s"] = time.perf_counter() - t0
    feats = np.stack([warmstart.features(grid, q["g"], q["g12"], q["Omega"], q["delta_slope"]) for q in prm])
    a = torch.from_numpy(feats).cuda()
    y = torch.from_numpy(np.stack([warmstart.to_channels(x) for x in gs])).cuda()
    f = sp.FNO(warmstart.CIN, warmstart.COUT, width=64, modes=32, layers=4, hidden=128, seed=1)
    rng = np.random.default_rng(WS_SEED)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(WS_ITERS):
        idx = torch.from_numpy(rng.choice(WS_TRAIN, WS_BATCH, replace=False)).cuda()
        losses.append(f.train_step(a[idx].contiguous(), y[idx].contiguous(), WS_LR))
    torch.cuda.synchronize()
    info.update(train_s=time.perf_counter() - t0, iters=WS_ITERS, batch=WS_BATCH, samples=WS_TRAIN,
                loss_first=float(np.mean(losses[:20])), loss_last=float(np.mean(losses[-20:])))
    return f, info


def warm_states(f, probs):
    """The model's proposals for the given sweep problems, normalised to one
    atom; (states, seconds including the host-side conversions)."""
    import torch
    from paper_2010_15069_gb300 import warmstart
    prm = inputs.sweep_params(len(probs), seed=3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = []
    for p, q in zip(probs, prm):
        g = p.grid
        a = torch.from_numpy(warmstart.features(g, q["g"], q["g12"], q["Omega"], q["delta_slope"])[None]).cuda()
        psi = warmstart.from_channels(f.forward(a).cpu().numpy()[0])
        nrm = g.dx * g.dy * float(np.sum(np.abs(psi) ** 2))
        out.append(psi / np.sqrt(nrm) if nrm > 0 else psi)
    return out, time.perf_counter() - t0


def ground_state_verdict(psi_a, psi_b, e_a, e_b, res_a, res_b, tol, gap_est=0.1, e_tol=1e-5):
    """The comparison of two relaxed ground states of the same problem
    (imaginary time can end on different metastable states of nearly equal
    energy from two starts): 'match' when both residuals are within tol and the states agree up
    to the global phase within tol / gap_est (the distance to the fixed point
    that a residual of tol allows for a slowest relaxation rate gap_est);
    'degenerate' when the energies agree within e_tol (relative) but the
    states do not (different metastable states of nearly equal energy, or a
    run not below tol); 'mismatch' otherwise.  Returns (verdict, max |dpsi|
    up to the phase, relative energy difference)."""
    ph = np.vdot(psi_b, psi_a)
    ph = ph / abs(ph) if abs(ph) > 0 else 1.0
    dpsi = float(np.abs(psi_a - psi_b * ph).max())
    de = abs(e_a - e_b) / max(abs(e_a), 1e-300)
    if res_a <= tol and res_b <= tol and dpsi <= tol / gap_est:
        return "match", dpsi, de
    if de <= e_tol:
        return "degenerate", dpsi, de
    return "mismatch", dpsi, de


def time_to_residual():
    """Wall time until the instances of one eighth of the sweep batch (8 x 256^2
    + 2 x 512^2 + 1 x 1024^2, the headline's generator) reach residual 1e-8,
    three ways:
      plain: the plain FP64 path (one complex128 context per instance, one
        after another, exact renormalisation, vortex-seeded);
      batched: one multi-size context, complex64 with the lagged
        renormalisation down to complex64's rounding floor, then complex128,
        converged instances frozen (vortex-seeded);
      warm: the same batched path started from the learned warm start's
        proposals (inference and conversions timed with it; the training on
        ground states of other parameter sets is reported apart).
    Every arm gives up an instance whose best residual has not halved in 40
    checks and has the same step budget per instance (the batched arms' two
    stages share it).  Times are charged over the instances all arms
    converge: the plain arm's per-instance times summed over them, and a
    second run of exactly those instances for each batched arm.  Per sampled
    converged instance: the energy and max |dpsi| (up to the global phase)
    between the plain and the warm arm and the FP64 oracle's residual of one
    exact step from the warm arm's result."""
    import torch
    import paper_2010_15069_gb300 as sp
    classes, probs, psi = sweep_problems(TTR_CLASSES)
    B = len(probs)
    plain = []
    for p, s in zip(probs, psi):
        g = p.grid
        with sp.Context(g.nx, g.ny, g.xmax, g.ymax, "c128") as c:
            c.set_potentials_separable(0, **p.separable, g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
            t = torch.from_numpy(s.copy()).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res, st = c.relax(t, SWEEP_DTAU, TTR_TOL, TTR_MAX, TTR_CHECK, give_up=True)
            el = time.perf_counter() - t0
            plain.append({"res": float(res[0]), "steps": int(st[1]), "s": el, "psi": t.cpu().numpy(),
                          "energy": float(c.energy(t)[0, 0])})

    def batched(idx, starts, extra_s=0.0):
        sub_probs = [probs[i] for i in idx]
        sub_psi = [starts[i] for i in idx]
        sub_classes = []
        for n, _ in TTR_CLASSES:
            k = sum(1 for p in sub_probs if p.grid.nx == n)
            if k:
                sub_classes.append((n, n, k, SWEEP_BOX, SWEEP_BOX))
        stream = torch.cuda.Stream()
        c, flat = make_multi(sub_classes, sub_probs, sub_psi, "c128", stream)
        with c:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res, st = c.relax(flat, SWEEP_DTAU, TTR_TOL, TTR_MAX, TTR_CHECK, ladder=True, give_up=True,
                              lagged=True)
            el = time.perf_counter() - t0 + extra_s
            en = c.energy(flat)[:, 0]
            views = [v.cpu().numpy() for v in c.class_views(flat)]
        states = [v[j] for v in views for j in range(v.shape[0])]
        return {"s": el, "res": res, "steps": st, "energy": en, "psi": states}

    cold = batched(list(range(B)), psi)
    f, train_info = train_warm_start()
    with f:
        wpsi, infer_s = warm_states(f, probs)
    if not all(np.isfinite(x).all() for x in wpsi):
        raise RuntimeError("the warm-start network proposed a non-finite spinor")
    warm = batched(list(range(B)), wpsi, infer_s)
    conv = {"plain": [i for i in range(B) if plain[i]["res"] <= TTR_TOL],
            "batched": [i for i in range(B) if cold["res"][i] <= TTR_TOL],
            "warm": [i for i in range(B) if warm["res"][i] <= TTR_TOL]}
    common = [i for i in range(B) if all(i in v for v in conv.values())]

    def rerun(run_all, starts, extra):
        if not common:
            return None
        if len(common) == B:
            return run_all["s"]
        return batched(common, starts, extra * len(common) / B)["s"]

    plain_s = sum(plain[i]["s"] for i in common)
    cold_s, warm_s = rerun(cold, psi, 0.0), rerun(warm, wpsi, infer_s)
    checks = []
    for cls_n in sorted({probs[i].grid.nx for i in common}):
        i = next(j for j in common if probs[j].grid.nx == cls_n)
        verdict, dpsi, de = ground_state_verdict(plain[i]["psi"], warm["psi"][i], plain[i]["energy"],
                                                 float(warm["energy"][i]), plain[i]["res"], float(warm["res"][i]),
                                                 TTR_TOL)
        checks.append({"instance": i, "grid": cls_n, "verdict_plain_vs_warm": verdict,
                       "rel_energy_diff_plain_vs_warm": de, "max_abs_dpsi_plain_vs_warm_up_to_phase": dpsi,
                       "oracle_one_step_residual": oracle_fixed_point_residual(probs[i], warm["psi"][i],
                                                                                SWEEP_DTAU)})
    verdicts = {}
    for i in common:
        v = ground_state_verdict(plain[i]["psi"], warm["psi"][i], plain[i]["energy"], float(warm["energy"][i]),
                                 plain[i]["res"], float(warm["res"][i]), TTR_TOL)[0]
        verdicts[v] = verdicts.get(v, 0) + 1
    return {"workload": "8 x 256^2 + 2 x 512^2 + 1 x 1024^2 instances of the sweep generator (seed 3), box "
                        f"[-12,12]^2, kL=1, dtau={SWEEP_DTAU:g}, residual checked every {TTR_CHECK} steps",
            "tol": TTR_TOL, "step_budget_per_instance": TTR_MAX,
            "arms": {"plain": "complex128, one context per instance in turn, exact renormalisation, 20-vortex seeded",
                     "batched": "one multi-size context: complex64 (lagged renormalisation) to its rounding "
                                "floor, then complex128 (lagged), converged instances frozen, 20-vortex seeded",
                     "warm": "the batched path from the warm-start network's proposals (inference timed)"},
            "converged": {k: len(v) for k, v in conv.items()} | {"all_arms": len(common), "of": B},
            "not_converged": {k: [i for i in range(B) if i not in v] for k, v in conv.items()},
            "seconds_over_common": {"plain_fp64_unbatched": plain_s, "batched": cold_s, "warm_batched": warm_s},
            "speedup_over_plain": {"batched": plain_s / cold_s if cold_s else None,
                                   "warm_batched": plain_s / warm_s if warm_s else None},
            "warm_inference_s": infer_s, "warm_start_training": train_info,
            "plain_steps_per_instance": [pl["steps"] for pl in plain],
            "batched_steps": {"complex64": int(cold["steps"][0]), "complex128": int(cold["steps"][1])},
            "warm_steps": {"complex64": int(warm["steps"][0]), "complex128": int(warm["steps"][1])},
            "all_instances_s": {"plain": sum(pl["s"] for pl in plain), "batched": cold["s"], "warm": warm["s"]},
            "verdicts_plain_vs_warm": verdicts, "checks": checks}


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
            torch.cuda.nvtx.range_push(f"single_timed_{n}")  # marks the timed run for profiler filters
            sec = timed(lambda k: c.step_real(t, DT, k), steps)
            torch.cuda.nvtx.range_pop()
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


C4_N, C4_STEPS = 2048, 10000


def config4_quench():
    """Config 4's large real-time run: one 2048^2 instance (box [-24, 24]^2,
    Omega = 2, detuning slope 0.2, g11 = g22 = 1000, g12 = 900, kL = 1): its
    ground state in the harmonic trap (relaxed in complex64 with the lagged
    renormalisation from a 20-vortex seeded state, seed 4, dtau = 2e-3, to
    residual 5e-3, above complex64's rounding floor 2^-18 / dtau, or a stall),
    then the trap quenched to omega = 1.1 and
    C4_STEPS real-time steps of dt = 5e-4 in one call, timed; the drift of the
    atom number and of the energy of the quenched Hamiltonian over the run
    (complex64).  The warm-start network is trained on the sweep's box
    [-12, 12]^2, so it is not used for this box."""
    import torch
    import paper_2010_15069_gb300 as sp
    n, L = C4_N, SINGLE_BOX
    kw = dict(Omega=2.0, delta_slope=0.2, g11=1000.0, g22=1000.0, g12=900.0, kL=1.0)
    p0 = inputs.problem(n, n, L, L, omega=1.0, **kw)
    p1 = inputs.problem(n, n, L, L, omega=1.1, **kw)
    stream = torch.cuda.Stream()
    peak, _ = peaks()
    with sp.Context(n, n, L, L, "c64", stream=stream) as c:
        c.set_potentials_separable(-1, **p0.separable, g11=p0.g11, g22=p0.g22, g12=p0.g12, kL=p0.kL)
        t = torch.from_numpy(inputs.vortex_spinor(p0.grid, n_vortices=20, radius=6.0, seed=4)
                             .astype(np.complex64)).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, st = c.relax(t, 2e-3, 5e-3, 20000, 250, give_up=True, lagged=True)
        relax_s = time.perf_counter() - t0
        c.set_potentials_separable(-1, **p1.separable, g11=p1.g11, g22=p1.g22, g12=p1.g12, kL=p1.kL)
        e0, n0 = c.energy(t)[0, 0], c.norm(t)[0].sum()
        c.autotune(t, DT)
        sec = timed_events(stream, lambda: c.step_real(t, DT, C4_STEPS))
        e1, n1 = c.energy(t)[0, 0], c.norm(t)[0].sum()
    return {"workload": f"{n}^2, box [-24,24]^2, Omega=2, delta=0.2y, g=1000, g12=900, kL=1, c64: ground state "
                        f"relaxed from 20 vortices, then the trap quenched omega 1 -> 1.1 and {C4_STEPS} real-time "
                        "steps of dt=5e-4 in one call",
            "ground_state": {"residual": float(res[0]), "steps": int(st[1]), "seconds": relax_s},
            "value": n * n * C4_STEPS / sec, "unit": "pt-steps/s", "ms_per_step": sec / C4_STEPS * 1e3,
            "step_frac": 64 * n * n * C4_STEPS / sec / 1e9 / peak,
            "l2_resident": 2 * n * n * 8 < L2_BYTES,
            "relative_drift": {"atom_number": float(abs(n1 - n0) / n0), "energy": float(abs(e1 - e0) / abs(e0))}}


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
    samples/s and the achieved rate of the network's algorithmic flops (training
    = 3 forward passes).  The pointwise channel products and the weight
    gradients run on the tcgen05 tensor cores (float32 operands split into
    bfloat16 terms: three MMA passes each); the truncated-DFT contractions
    and the per-mode mixing run on the CUDA cores."""
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
            "achieved_tflops": flop / sec / 1e12,
            "where": "channel products and weight gradients on tcgen05 tensor cores; truncated DFTs and mode "
                     "mixing on CUDA cores"}


# ------------------------------------------------------------- CPU oracle

def oracle_instance(i=0):
    """The FP64 oracle's model and initial spinor of sweep instance i (256^2)."""
    import oracle
    _, probs, psi = sweep_problems([(256, i + 1)])
    p = probs[i]
    g = p.grid
    m = oracle.Model(g.nx, g.ny, g.xmax, g.ymax, V=p.V, delta=p.delta, Omega=p.Omega,
                     g11=p.g11, g22=p.g22, g12=p.g12, kL=p.kL)
    return m, psi[i], g.nx * g.ny


def oracle_rate(budget_s=12.0, max_steps=2000):
    """The FP64 oracle on the first 256^2 instance of the sweep (imaginary time,
    exact renormalisation, one thread): (pt-steps/s, steps, seconds)."""
    m, psi, npt = oracle_instance(0)
    t0 = time.perf_counter()
    psi = m.step(psi, SWEEP_DTAU, 1, imag=True)
    one = time.perf_counter() - t0
    n = int(max(1, min(max_steps, budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    m.step(psi, SWEEP_DTAU, n, imag=True)
    dt = time.perf_counter() - t0
    return npt * n / dt, n, dt


def _oracle_worker(i, budget_s):
    """One pool worker: oracle imaginary-time steps on sweep instance i for about budget_s."""
    m, psi, npt = oracle_instance(i)
    psi = m.step(psi, SWEEP_DTAU, 1, imag=True)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        psi = m.step(psi, SWEEP_DTAU, 10, imag=True)
        n += 10
    return npt * n, time.perf_counter() - t0


def oracle_rate_all_cores(budget_s=8.0):
    """The same oracle, one independent 256^2 sweep instance per host core in a
    spawned process pool (the oracle itself is single-threaded and unchanged):
    (aggregate pt-steps/s, workers, seconds)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_worker, [(i, budget_s) for i in range(cores)])
    wall = time.perf_counter() - t0
    return sum(r[0] / r[1] for r in res), cores, wall


def copy_ceiling(t, reps=7):
    """Pinned host <-> device copy rates of one batch-sized buffer, GB/s: in
    alone, out alone, and both directions at once on two streams (the bound
    of an end-to-end step that moves the batch in and out); each the fastest
    of `reps` timed repetitions."""
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
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return best

    t_in, t_out = timed(h2d), timed(d2h)
    t_both = timed(lambda: (h2d(), d2h()))
    return {"h2d_gbs": nbytes / t_in / 1e9, "d2h_gbs": nbytes / t_out / 1e9,
            "both_directions_gbs": 2 * nbytes / t_both / 1e9, "bytes": nbytes}


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


def bf16_peaks():
    """The sustained dense bfloat16 rate of MEASURED_PEAKS.json (TFLOP/s), or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"])
    except (OSError, KeyError, ValueError):
        return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ arms

def sweep_config(dtype, choice=None, tune_ms=None, chosen_by="auto", renorm="lagged"):
    cls = [{"grid": [n, n], "instances": k} for n, k in SWEEP_CLASSES]
    out = {"workload": "imaginary-time parameter-sweep batch 64 x 256^2 + 16 x 512^2 + 4 x 1024^2 (12.58 M points "
                       f"per component), box [-12,12]^2, kL=1, sweep generator (seed 3), 20-vortex seeded, "
                       f"dtau={SWEEP_DTAU:g}, {dtype}, {renorm} renormalisation",
           "classes": cls, "dtau": SWEEP_DTAU, "box": [-SWEEP_BOX, SWEEP_BOX],
           "l2": "batch larger than L2 (no flush)", "parallelism": "instances sharded per GPU (one batch per GPU)"}
    if choice is not None:
        names = ["plain", "persistent TMA", "warp-local TMA"]
        out["schedule"] = {"per_class": [{"grid": n, "persistent_row": bool(v & 1), "column_pass": names[int(v) >> 1]}
                                         for (n, _), v in zip(SWEEP_CLASSES, choice)],
                           "chosen_by": chosen_by,
                           "autotune_ms_per_step": [float(x) for x in tune_ms] if tune_ms is not None else None}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    m, psi, npt = oracle_instance(0)
    psi = m.step(psi, SWEEP_DTAU, args.warmup, imag=True)
    t0 = time.perf_counter()
    m.step(psi, SWEEP_DTAU, args.steps, imag=True)
    el = time.perf_counter() - t0
    value = npt * args.steps / el
    line = {
        "impl": "reference", "metric": "grid-point-steps/s", "value": value, "unit": "pt-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": sweep_config("f64 (oracle)", renorm="exact"),
        "cpu_baseline": {"value": value, "unit": "pt-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"the first 256x256 instance of the sweep batch, {args.steps} FP64 imaginary-time "
                                   "steps (exact renormalisation), one thread"},
        "e2e": {"value": value, "unit": "pt-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def realtime_batch(args, stream, dist, world, rank, peak, peak_kind):
    """The real-time batch of the 256^2 problem (256 instances, complex64): K
    steps in one call, the roofline of its dominant pass, and the cuFFT
    comparator (the paper's step structure) on the same batch."""
    import torch
    B, dtype = args.instances, "c64"
    first, _ = instance_range(rank, world, B)
    c, t, _ = make_workload(B, dtype, stream=stream, first=first)
    pts = B * NX * NY
    if args.schedule == "auto":
        choice, _ = c.autotune(t, DT)
    else:
        choice = np.array([{"persistent": 3, "warp": 5, "plain": 0}[args.schedule]])
    c.step_real(t, DT, args.warmup)
    steps = args.steps
    if dist is not None:
        dist.barrier()
    torch.cuda.nvtx.range_push("realtime_timed")
    sec = max_over_ranks(timed_events(stream, lambda: c.step_real(t, DT, steps)), dist, "cuda")
    torch.cuda.nvtx.range_pop()
    c.set_timing(True)
    c.step_real(t, DT, steps)
    kt = c.timing()
    c.set_timing(False)
    kinds = {k: v for k, v in kt.items() if k.startswith(("row_real_fused", "col_real"))}
    dom = max(kinds, key=lambda k: kinds[k][1])
    n_dom, ms_dom = kinds[dom]
    avg_s = ms_dom * 1e-3 / n_dom
    alg_bytes = BYTES_PER_PT_PASS[dtype] * pts
    achieved = alg_bytes / avg_s / 1e9
    c.cufft_step_real(t, DT, 3)
    if dist is not None:
        dist.barrier()
    sec_ref = max_over_ranks(timed_events(stream, lambda: c.cufft_step_real(t, DT, CUFFT_STEPS)), dist, "cuda")
    c.close()
    value = world * pts * steps / sec
    return {"workload": f"256x256 real-time two-component GPE x {B} instances (Omega=2, delta=0.5y, kL=1, g=200, "
                        f"dt=5e-4), c64, each the 64^2 ground state upsampled with seeded phase noise",
            "value": value, "unit": "pt-steps/s", "steps": steps, "ms_per_step": sec / steps * 1e3,
            "schedule": {"persistent_row": bool(choice[0] & 1),
                         "column_pass": ["plain", "persistent TMA", "warp-local TMA"][int(choice[0]) >> 1]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": measured_traffic(f"{dom}:{dtype}:{B}"), "kernel": dom,
                         "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_s * 1e3,
                         "peak_source": peak_kind,
                         "step_frac": PASSES_PER_STEP * alg_bytes * steps / sec / 1e9 / peak},
            "kernel_ms": {k: {"launches": v[0], "avg_ms": v[1] / v[0]} for k, v in kt.items()},
            "cufft_comparator": {"value": world * pts * CUFFT_STEPS / sec_ref, "unit": "pt-steps/s",
                                 "steps": CUFFT_STEPS,
                                 "what": "same batch and dt, cuFFT 2D C2C transforms + separate R and K kernels "
                                         "(the paper's step structure)",
                                 "fused_over_cufft": value / (world * pts * CUFFT_STEPS / sec_ref)}}


def run_fused(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    total = sum(k for _, k in SWEEP_CLASSES)
    first, _ = instance_range(rank, world, total)
    classes, probs, psi = sweep_problems(SWEEP_CLASSES, first)
    pts = sum(n * n * k for n, k in SWEEP_CLASSES)
    c, flat = make_multi(classes, probs, psi, "c64", stream)
    if args.schedule == "auto":
        # the library's autotuner picks the pass variants per size class (scratch copy; psi unchanged)
        choice, tune_ms = c.autotune(flat, 5e-4)
    else:
        code = {"persistent": 3, "warp": 5, "plain": 0}[args.schedule]
        choice, tune_ms = np.array([code] * len(SWEEP_CLASSES)), None

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up, then the timed region: K steps in one call
    c.step_imag(flat, SWEEP_DTAU, args.warmup, lagged=True)
    barrier()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        torch.cuda.nvtx.range_push("sweep_timed")  # marks the timed region for profiler filters
        start.record(stream)
        c.step_imag(flat, SWEEP_DTAU, args.steps, lagged=True)
        stop.record(stream)
        launches = c.last_launches()
        barrier()
        torch.cuda.nvtx.range_pop()
    ms = max_over_ranks(start.elapsed_time(stop), dist, "cuda")
    value = world * pts * args.steps / (ms * 1e-3)
    peak, peak_kind = peaks()
    psi_bytes = flat.numel() * flat.element_size()

    # per-kernel event times, each size class alone (see kernel_times_in_turn)
    tsteps = min(args.steps, TIMING_STEPS)
    per = kernel_times_in_turn(c, flat, classes, probs, "c64", stream, tsteps, True)
    n_dom, k_dom, kind, cnt, ms_dom = dominant(per)
    avg_s = ms_dom * 1e-3 / cnt
    alg_bytes = BYTES_PER_PT_PASS["c64"] * n_dom * n_dom * k_dom
    achieved = alg_bytes / avg_s / 1e9

    # the exact renormalisation (three passes per step) on the same batch
    c.step_imag(flat, SWEEP_DTAU, 3)
    barrier()
    sec_exact = max_over_ranks(timed_events(stream, lambda: c.step_imag(flat, SWEEP_DTAU, tsteps)), dist, "cuda")

    # end to end through the C ABI with pinned host buffers: every step copies
    # the batch in, steps it once and copies it back
    host = torch.empty(tuple(flat.shape), dtype=flat.dtype, pin_memory=True)
    host.copy_(flat)
    hnp = host.numpy()
    c.step_imag(hnp, SWEEP_DTAU, 1)
    e2e_steps = max(3, min(args.steps, 20))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        c.step_imag(hnp, SWEEP_DTAU, 1)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    barrier()
    ceiling = copy_ceiling(flat)
    c.close()
    del flat, host

    ceil = ceilings() if world == 1 else None
    fp64_peak = ceil.get("fp64_fma_tflops") if isinstance(ceil, dict) else None

    # the same workload in complex128 (FP64 operators): its own roofline
    c2, flat2 = make_multi(classes, probs, psi, "c128", stream)
    c2.autotune(flat2, 5e-4)
    c2.step_imag(flat2, SWEEP_DTAU, 3, lagged=True)
    barrier()
    k128 = min(args.steps, C128_STEPS)
    sec128 = max_over_ranks(timed_events(stream, lambda: c2.step_imag(flat2, SWEEP_DTAU, k128, lagged=True)), dist,
                            "cuda")
    per128 = kernel_times_in_turn(c2, flat2, classes, probs, "c128", stream, k128, True)
    c2.close()
    del flat2
    n8, k8, kind8, cnt8, ms8 = dominant(per128)
    avg8 = ms8 * 1e-3 / cnt8
    flops8 = flops_per_point(kind8, n8) * n8 * n8 * k8
    bytes8 = BYTES_PER_PT_PASS["c128"] * n8 * n8 * k8
    c128 = {"value": world * pts * k128 / sec128, "unit": "pt-steps/s", "steps": k128,
            "ms_per_step": sec128 / k128 * 1e3, "dtype": "f64", "renormalisation": "lagged",
            "roofline": {"bound": "alu", "unit": "TFLOP/s", "kernel": f"{kind8} {n8}^2 x {k8}",
                         "achieved": flops8 / avg8 / 1e12, "peak": fp64_peak,
                         "frac": flops8 / avg8 / 1e12 / fp64_peak if fp64_peak else None,
                         "algorithmic_flops_per_launch": flops8, "avg_launch_ms": avg8 * 1e3,
                         "peak_source": "measured: FP64 fma microbenchmark (spgpe_probe_ceilings)",
                         "hbm_frac": bytes8 / avg8 / 1e9 / peak},
            "kernel_ms_by_class": [{"grid": n, "instances": k, "kernels": {kk: {"launches": v[0], "avg_ms": v[1] / v[0]}
                                                                            for kk, v in kt.items()}}
                                   for n, k, kt in per128]}

    rt = realtime_batch(args, stream, dist, world, rank, peak, peak_kind) if args.realtime else None

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = cpu_all = None
    if world == 1:
        rate, n, el = oracle_rate()
        cpu = {"value": rate, "unit": "pt-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"the first 256x256 instance of the sweep batch, {n} FP64 imaginary-time steps in "
                         f"{el:.1f} s (exact renormalisation, one thread)"}
        rate, cores, el = oracle_rate_all_cores()
        cpu_all = {"value": rate, "unit": "pt-steps/s", "cores": cores, "kind": "oracle",
                   "sample": f"one 256x256 sweep instance per core, FP64 imaginary-time steps for about 8 s each "
                             f"({el:.1f} s wall), spawned process pool"}
    line = {
        "metric": "grid-point-steps/s", "value": value, "unit": "pt-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": sweep_config("c64", choice, tune_ms, args.schedule),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(f"{kind}:c64:{n_dom}x{k_dom}"),
                     "kernel": f"{kind} {n_dom}^2 x {k_dom}",
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_s * 1e3,
                     "peak_source": peak_kind,
                     "kernel_timing": f"{tsteps} steps of each size class alone on the GPU (classes in turn)",
                     "step_frac": 64 * pts * args.steps / (ms * 1e-3) / 1e9 / peak},
        "kernel_ms_by_class": [{"grid": n, "instances": k, "kernels": {kk: {"launches": v[0], "avg_ms": v[1] / v[0]}
                                                                        for kk, v in kt.items()}}
                               for n, k, kt in per],
        "exact_renormalisation": {"value": world * pts * tsteps / sec_exact, "unit": "pt-steps/s", "steps": tsteps,
                                  "ms_per_step": sec_exact / tsteps * 1e3, "bytes_per_pt_step": 96,
                                  "step_frac": 96 * pts * tsteps / sec_exact / 1e9 / peak},
        "c128": c128,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "e2e": {"value": world * pts * e2e_steps / e2e_s, "unit": "pt-steps/s", "h2d_bytes_per_step": psi_bytes,
                "d2h_bytes_per_step": psi_bytes, "steps": e2e_steps,
                "what": "spgpe_step_imag on pinned host buffers, one step per call (exact renormalisation)",
                "copy_gbs": 2 * psi_bytes * e2e_steps / e2e_s / 1e9, "copy_ceiling": ceiling,
                "frac_of_copy_ceiling": 2 * psi_bytes * e2e_steps / e2e_s / 1e9 / ceiling["both_directions_gbs"]},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "ceilings": dict(ceil, l2_capacity_mib_estimate=l2_capacity_mib(ceil)) if isinstance(ceil, dict) else ceil,
    }
    if rt is not None:
        line["realtime_batch"] = rt
    # the secondary measurements: a failure in one is recorded in its place
    def secondary(fn):
        try:
            return fn()
        except Exception as e:  # noqa: BLE001 - the headline line is printed regardless
            log(f"secondary measurement failed: {e!r}")
            return {"error": repr(e)}
    if world == 1 and args.ttr:
        line["time_to_residual"] = secondary(time_to_residual)
    if world == 1 and args.single:
        line["single_instance"] = secondary(lambda: single_instance(args.single_steps, tune=args.schedule == "auto"))
        line["config4_quench"] = secondary(config4_quench)
    if world == 1 and args.fno:
        fn = fno_throughput()
        bf16 = bf16_peaks()
        fp32 = ceil.get("fp32_fma_tflops") if isinstance(ceil, dict) else None
        fn.update(frac_of_bf16_tensor_sustained=fn["achieved_tflops"] / bf16 if bf16 else None,
                  bf16_tensor_sustained_tflops=bf16,
                  frac_of_fp32_fma=fn["achieved_tflops"] / fp32 if fp32 else None, fp32_fma_tflops=fp32,
                  peak_source="MEASURED_PEAKS.json bf16_tflops_sustained; FP32 fma from spgpe_probe_ceilings")
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
    ap.add_argument("--instances", type=int, default=DEFAULT_INSTANCES,
                    help="instances of the real-time 256^2 batch")
    ap.add_argument("--schedule", choices=["auto", "persistent", "warp", "plain"], default="auto",
                    help="pass variants: autotuned (default) or fixed")
    ap.add_argument("--realtime", type=int, default=1, help="1: also time the real-time 256^2 batch (0: skip)")
    ap.add_argument("--single", type=int, default=1,
                    help="1: also time one 2048^2 and one 4096^2 instance against the cuFFT comparator (0: skip)")
    ap.add_argument("--single-steps", type=int, default=200, help="timed steps of each single-instance run")
    ap.add_argument("--fno", type=int, default=1, help="1: also time training of the warm-start FNO (0: skip)")
    ap.add_argument("--ttr", type=int, default=1, help="1: also run the time-to-residual comparison (0: skip)")
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
