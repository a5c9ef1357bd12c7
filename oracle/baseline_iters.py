"""Oracle iterations per solve for the benchmark workload (writes baseline_iters.json).

The CPU baseline of bench.py times a bounded number of oracle BiCGStab
iterations on the host and converts that rate to solves/s with the number of
iterations the oracle itself needs per solve of the same systems. This script
computes those counts with the oracle only (full unpreconditioned BiCGStab to
relative residual 1e-8) and stores them next to it.

Workload: 16^3x32 lattice, smoothed links U = exp(i 0.4 H) (gauge seed 1003),
m = -0.35, shifts {0.005, 0.03, 0.15, 0.6}, Z4 noise (seed 2003, job 0,
level l, sample 0).
"""

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import inputs  # noqa: E402
from oracle import philox, solve  # noqa: E402

DIMS = (16, 16, 16, 32)
M = -0.35
SIGMAS = [0.005, 0.03, 0.15, 0.6]


def main():
    u = inputs.gauge_field(DIMS, "smooth", seed=1003, eps=0.4)
    v = int(np.prod(DIMS))
    out = {"workload": "16^3x32 eps=0.4 gauge_seed=1003 m=-0.35", "tol": 1e-8, "iters": {}, "seconds": {}}
    for lev, s in enumerate(SIGMAS):
        z = philox.z4_noise(v, 2003, 0, lev, 0)
        t = time.time()
        r = solve.shifted_solve(u, z, M, s, DIMS, -1, tol=1e-8, max_iter=20000)
        out["iters"][repr(s)] = int(r.iters)
        out["seconds"][repr(s)] = time.time() - t
        print(s, r.iters, r.rel_resid, time.time() - t, flush=True)
    with open(os.path.join(HERE, "baseline_iters.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
