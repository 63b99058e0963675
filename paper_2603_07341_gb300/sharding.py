"""Realisation sharding of a static-disorder ensemble over ranks.

The realisations of an ensemble are independent problems (each is its own
single-exciton Holstein model with its own site energies), and the quantity the
paper takes from such runs is the disorder-averaged autocorrelation
C(t) = (1/R) sum_r C_r(t), C_r(t) = <psi(0)|psi_r(t)> (the aggregates section:
the absorption spectrum is the damped Fourier transform of the averaged
signal).  So the ensemble splits across ranks with no exchange while it runs:
rank k evolves realisations [lo_k, hi_k) as one batched handle, and the only
collective is a single all-reduce (sum) of sum_r C_r(t) over the steps at the
end; the spectrum is taken from the reduced mean on every rank.

run_sharded_ensemble() is the driver; the work of a slice is a callable so the
same host logic runs with the CUDA library (gpu_slice_runner) or, in the
multi-process CPU tests, with any other implementation.
"""
from __future__ import annotations

import numpy as np


def shard_range(R: int, world: int, rank: int):
    """Contiguous, balanced block of realisations for `rank` of `world`:
    the first R % world ranks take one more."""
    if R < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("bad shard request")
    base, extra = divmod(R, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def run_sharded_ensemble(R, nsteps, run_slice, group=None, device=None):
    """Evolve realisations 0..R-1 split over the ranks of `group` (torch
    process group; None = single process).

    run_slice(lo, hi) -> complex array [nsteps + 1, hi - lo] of C_r(t_k) for
    the realisations lo..hi-1 (k = 0 is psi(0)), or None for an empty slice.
    Returns (C_mean [nsteps + 1] complex, the disorder average over all R,
    identical on every rank; (lo, hi) of this rank; the local C_r block)."""
    world, rank = 1, 0
    dist = None
    if group is not None or _dist_ready():
        import torch.distributed as dist
        world = dist.get_world_size(group)
        rank = dist.get_rank(group)
    lo, hi = shard_range(R, world, rank)
    C_loc = run_slice(lo, hi) if hi > lo else None
    s = np.zeros((nsteps + 1, 2), dtype=np.float64)
    if C_loc is not None:
        C_loc = np.asarray(C_loc, dtype=np.complex128).reshape(nsteps + 1, hi - lo)
        tot = C_loc.sum(axis=1)
        s[:, 0], s[:, 1] = tot.real, tot.imag
    if dist is not None and world > 1:
        import torch
        t = torch.from_numpy(s)
        if device is not None:
            t = t.to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        s = t.cpu().numpy()
    return (s[:, 0] + 1j * s[:, 1]) / R, (lo, hi), C_loc


def _dist_ready():
    try:
        import torch.distributed as dist
        return dist.is_available() and dist.is_initialized()
    except Exception:
        return False


def gpu_slice_runner(model, eps_all, start_state, dt, theta, nsteps, precision=None):
    """run_slice for the CUDA library: one batched handle (batch = hi - lo,
    site energies eps_all[lo:hi]) on the current device, nsteps steps, the
    per-realisation C_r(t) read from its observables records."""
    from . import binding as B

    def run(lo, hi):
        m = dict(model)
        m["batch"] = hi - lo
        m["eps"] = np.ascontiguousarray(np.asarray(eps_all)[lo:hi])
        if precision is not None:
            m["precision"] = precision
        sol = B.Solver(**m)
        try:
            sol.set_state(*start_state)
            sol.step(dt, nsteps, theta)
            rec = sol.observables(0, nsteps + 1)
            N = int(model["n_sites"])
            if hi - lo == 1:
                return (rec[:, 4] + 1j * rec[:, 5]).reshape(-1, 1)
            return B.records_dict(rec, N, hi - lo)["C_r"]
        finally:
            sol.close()

    return run
