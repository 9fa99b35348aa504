"""Process-pool jobs of the oracle for full-size comparisons (test infrastructure only).

Each job rebuilds the seeded workload in the worker (nothing large is pickled)
and returns one shot's Born traces, or one shot's Born traces and their
migration, or one shot's terms of the 3D preconditioning pipeline on a reduced
grid.  Start pools with the ``spawn`` method.
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


def born_adjoint_shot(spec):
    """spec = (config, shape, nt, ns, pad, p, shot): on a reduced grid of the configuration's
    recipe, one shot's terms F_s^T F_s y_j of the p trial functions y_j and F_s^T F_s dm_ref of
    the reference perturbation, stacked as (p + 1, *shape) (the preconditioning pipeline of the
    3D configuration: fit on H y_j, then precondition the migrated data F^T F dm_ref)."""
    from workloads import mini_config

    from .wave import problem_from_workload
    cfg, shape, nt, ns, pad, p, shot = spec
    wl = mini_config(cfg, shape=shape, nt=nt, ns=ns, pad=pad, p=p)
    prob = problem_from_workload(wl)
    dms = np.concatenate([wl.trials, wl.extra["dm_ref"][None]]).astype(np.float64)
    d = prob.born(shot, dms)
    return np.stack([prob.adjoint(shot, d[b]) for b in range(p + 1)])


def start_pool(specs, workers=None, fn=None):
    """Start the jobs (run_job, or fn) asynchronously in a spawn pool; returns (pool, AsyncResult)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(workers or len(specs))
    return pool, pool.map_async(fn or run_job, specs)
