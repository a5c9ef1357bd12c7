"""Oracle iterations per solve for the benchmark workload (writes baseline_iters.json).

The CPU baseline of bench.py times a bounded number of oracle BiCGStab
iterations on the host and converts that rate to solves/s with the number of
iterations the oracle itself needs per solve of the same systems. This script
computes those counts with the oracle only (full unpreconditioned BiCGStab to
relative residual 1e-8) and stores them next to it.

Workloads (keys of the JSON file):
  16x32  16^3x32, smoothed links U = exp(i 0.4 H) (gauge seed 1003), m = -0.35,
         shifts {0.005, 0.03, 0.15, 0.6}, Z4 noise seed 2003
  8x8    8^4, U = exp(i 0.3 H) (gauge seed 1002), m = -0.2, shifts {0.02, 0.1, 0.5},
         Z4 noise seed 2002
each solved for the noise vector (job 0, level l, sample 0).
Usage: python oracle/baseline_iters.py [workload ...]
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

WORKLOADS = {
    "16x32": dict(dims=(16, 16, 16, 32), eps=0.4, gauge_seed=1003, noise_seed=2003, m=-0.35,
                  sigmas=[0.005, 0.03, 0.15, 0.6]),
    "8x8": dict(dims=(8, 8, 8, 8), eps=0.3, gauge_seed=1002, noise_seed=2002, m=-0.2, sigmas=[0.02, 0.1, 0.5]),
}
PATH = os.path.join(HERE, "baseline_iters.json")


def calibrate(name):
    w = WORKLOADS[name]
    dims = w["dims"]
    u = inputs.gauge_field(dims, "smooth", seed=w["gauge_seed"], eps=w["eps"])
    v = int(np.prod(dims))
    out = {"tol": 1e-8, "iters": {}, "seconds": {}}
    for lev, s in enumerate(w["sigmas"]):
        z = philox.z4_noise(v, w["noise_seed"], 0, lev, 0)
        t = time.time()
        r = solve.shifted_solve(u, z, w["m"], s, dims, -1, tol=1e-8, max_iter=20000)
        out["iters"][repr(s)] = int(r.iters)
        out["seconds"][repr(s)] = time.time() - t
        print(name, s, r.iters, r.rel_resid, time.time() - t, flush=True)
    return out


def main(names):
    data = {}
    if os.path.exists(PATH):
        with open(PATH) as f:
            data = json.load(f)
        if "iters" in data:  # single-workload layout of an earlier run
            data = {"16x32": data}
    for n in names:
        data[n] = calibrate(n)
    with open(PATH, "w") as f:
        json.dump(data, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or sorted(WORKLOADS))
