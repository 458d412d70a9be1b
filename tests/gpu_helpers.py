"""Shared helpers of the GPU parity tests: build a librrmhd context from a
workload, and run the oracle on the same instances."""
import numpy as np

import oracle as O
from paper_2212_00370_gb300 import rrmhd


def oracle_params(w, **kw):
    return O.Params(gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl, **kw)


def oracle_grid(g):
    nd = g["ndim"]
    return O.Grid(nd, tuple(g["n"][:nd]), tuple(g["dx"][:nd]), tuple(g["bc"][:nd]))


def gpu_context(w, **opts):
    import torch
    grids = [rrmhd.make_grid(g["ndim"], g["n"], g["dx"], g["bc"]) for g in w.grids]
    ctx = rrmhd.Context(grids, gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl, **opts)
    ctx.set_opacity(torch.tensor(w.kappa, device="cuda"), torch.tensor(w.sigma, device="cuda"))
    ctx.set_state(torch.tensor(w.V, device="cuda"))
    ctx.set_times(np.zeros(w.n_inst), w.t_end)
    return ctx


def oracle_run_instance(w, i, nsteps, P=None):
    """Advance instance i of workload w by up to nsteps steps (to t_end).
    Returns (U, V, t, steps, nfail)."""
    g, V, kappa, sigma = w.instance(i)
    P = P or oracle_params(w)
    V = np.ascontiguousarray(V).copy()
    U = O.prim2con(V, P)
    t, steps, nfail = O.run(oracle_grid(g), 0.0, float(w.t_end[i]), U, V, kappa, sigma, P,
                            max_steps=nsteps)
    return U, V, t, steps, nfail


def compare_bitwise(a, b, what):
    """Exact equality, with a readable summary of the first differences."""
    a = np.asarray(a)
    b = np.asarray(b)
    if np.array_equal(a, b):
        return
    diff = a != b
    idx = np.argwhere(diff)[:5]
    scale = np.maximum(np.abs(a), np.abs(b))
    rel = np.where(diff, np.abs(a - b) / np.where(scale > 0, scale, 1), 0)
    raise AssertionError(f"{what}: {diff.sum()} of {diff.size} values differ; max rel "
                         f"{rel.max():.3e}; first at {idx.tolist()}")


def _oracle_job(job):
    """Worker of oracle_pool_runs: (n, dx, V, kappa, sigma, gamma, a_rad, cfl, t_end,
    max_steps) of one 1D outflow instance -> (U, V, t, steps, nfail)."""
    n, dx, V, kappa, sigma, gamma, a_rad, cfl, t_end, max_steps = job
    P = O.Params(gamma=gamma, a_rad=a_rad, cfl=cfl)
    V = np.ascontiguousarray(V, dtype=np.float64).copy()
    U = O.prim2con(V, P)
    t, steps, nfail = O.run(O.Grid(1, (int(n),), (float(dx),)), 0.0, float(t_end), U, V,
                            np.ascontiguousarray(kappa), np.ascontiguousarray(sigma), P,
                            max_steps=int(max_steps))
    return U, V, t, steps, nfail


def oracle_pool_runs(jobs, processes=None):
    """Run oracle jobs (see _oracle_job) in a spawn pool (safe after CUDA is initialised)."""
    import multiprocessing as mp
    import os
    processes = processes or min(len(jobs), os.cpu_count() or 1, 32)
    with mp.get_context("spawn").Pool(processes) as pool:
        return pool.map(_oracle_job, jobs, chunksize=1)
