"""Oracle runs of the large parity cases in spawned worker processes.

A job is a dict: grid (nx, ny, xmax, ymax), the 2D potentials V, delta, Omega
(None for zero), couplings g11, g22, g12, kL, the initial spinor psi, the time
step dt, the number of steps n, imag, norm mode and target, and whether the
last-step residual is wanted.  run() returns (spinor, energy terms,
residual or None).  The workers run the oracle unchanged; the pool only lets
the independent cases of one test module use the host's cores side by side.
"""
import multiprocessing as mp
import os


def run(job):
    import oracle
    nx, ny, xmax, ymax = job["grid"]
    m = oracle.Model(nx, ny, xmax, ymax, V=job["V"], delta=job.get("delta"), Omega=job.get("Omega"),
                     g11=job["g11"], g22=job["g22"], g12=job["g12"], kL=job["kL"])
    res = None
    if job.get("residual"):
        psi, res = m.step(job["psi"], job["dt"], job["n"], imag=job["imag"], norm_mode=job.get("mode", 0),
                          target=job.get("target", (0.5, 0.5)), residual=True)
    else:
        psi = m.step(job["psi"], job["dt"], job["n"], imag=job["imag"], norm_mode=job.get("mode", 0),
                     target=job.get("target", (0.5, 0.5)))
    return psi, m.energy(psi), res


def job_for(p, psi, dt, n, imag=True, mode=0, target=(0.5, 0.5), residual=False):
    """A job for the problem p (paper_2010_15069_gb300.inputs.Problem)."""
    g = p.grid
    return dict(grid=(g.nx, g.ny, g.xmax, g.ymax), V=p.V, delta=p.delta, Omega=p.Omega, g11=p.g11, g22=p.g22,
                g12=p.g12, kL=p.kL, psi=psi, dt=dt, n=n, imag=imag, mode=mode, target=target, residual=residual)


def run_all(jobs):
    """Run the jobs in a spawned process pool (at most one per host core)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(max(1, min(len(jobs), cores))) as pool:
        return pool.map(run, jobs)
