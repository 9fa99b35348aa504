"""Writes tests/golden/oracle_small2d.json from the oracle alone (no GPU code is imported).

A small 2D problem of the configuration-1 recipe (24 x 26 interior, pad 6, nt 160,
2 shots): sampled Born traces (Sec. 2 linearised wave equation), sampled values and
the norm of H dm = F*F dm (Sec. 1.1), and both sides of the dot-product test.  The
stored values pin the oracle against its own later edits: a change of its
arithmetic must come with a regenerated file and, in the commit message, the
passage that justifies it.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.wave import problem_from_workload  # noqa: E402
from workloads import mini_config  # noqa: E402

SPEC = dict(config=1, shape=(24, 26), nt=160, ns=2, pad=6)
TRACE_SAMPLES = [(0, 40, 3), (0, 120, 12), (1, 80, 20), (1, 159, 25)]   # (shot, n, receiver)
MODEL_SAMPLES = [(3, 4), (12, 13), (20, 22)]                           # interior (z, x)


def compute():
    wl = mini_config(SPEC["config"], shape=SPEC["shape"], nt=SPEC["nt"], ns=SPEC["ns"], pad=SPEC["pad"])
    p = problem_from_workload(wl)
    dm = wl.trials[0].astype(np.float64)
    d = [p.born(s, dm) for s in range(p.ns)]
    hdm = sum(p.adjoint(s, d[s]) for s in range(p.ns))
    r = np.random.default_rng(7).standard_normal((p.ns, p.nt, p.nr))
    fr = sum(p.adjoint(s, r[s]) for s in range(p.ns))
    return {
        "spec": {k: (list(v) if isinstance(v, tuple) else v) for k, v in SPEC.items()},
        "born_samples": [[s, n, j, float(d[s][n, j])] for s, n, j in TRACE_SAMPLES],
        "born_norm": float(np.sqrt(sum(np.sum(x ** 2) for x in d))),
        "hdm_samples": [[z, x, float(hdm[z, x])] for z, x in MODEL_SAMPLES],
        "hdm_norm": float(np.linalg.norm(hdm)),
        "dot_Fdm_r": float(sum(np.vdot(d[s], r[s]) for s in range(p.ns))),
        "dot_dm_Fadj_r": float(np.vdot(dm, fr)),
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "oracle_small2d.json")
    with open(out, "w") as f:
        json.dump(compute(), f, indent=1)
    print(out)
