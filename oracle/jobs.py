"""Process-pool jobs of the oracle for full-size comparisons (test infrastructure only).

Each job rebuilds the seeded workload in the worker (nothing large is pickled)
and returns one shot's Born traces, or one shot's Born traces and their
migration.  Start pools with the ``spawn`` method.
"""
from __future__ import annotations

import numpy as np


def run_job(spec):
    """spec = (config, kind, shot, ckpt): kind 'born' -> traces; 'born+adj' -> (traces, image)."""
    from workloads import make_config

    from .wave import problem_from_workload
    cfg, kind, shot, ckpt = spec
    wl = make_config(cfg)
    prob = problem_from_workload(wl)
    dm = wl.trials[0].astype(np.float64)
    d = prob.born(shot, dm)
    if kind == "born":
        return d
    return d, prob.adjoint(shot, d, ckpt=ckpt)


def start_pool(specs, workers=None):
    """Start the jobs asynchronously in a spawn pool; returns (pool, AsyncResult)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(workers or len(specs))
    return pool, pool.map_async(run_job, specs)
