"""bench.py's CPU baselines: the oracle timed on one core and on several at once.

The all-core figure comes from spawned single-threaded workers, each timing the one-core
sample on its own system after a common barrier; the pool's rate is the sum of theirs.
Short samples on the 8^4 workload keep this test to a few seconds.
"""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_one_core_sample():
    w = bench.WORKLOADS["8x8"]
    rate, sample, dt = bench.oracle_rate(w, 0.3)
    assert rate > 0 and dt > 0
    assert "oracle BiCGStab iterations" in sample


def test_pool_sums_its_workers_and_is_reused():
    w = bench.WORKLOADS["8x8"]
    one, _, _ = bench.oracle_rate(w, 0.3)
    pool = bench.OraclePool(w, n=2)
    try:
        first, longest = pool.rate(0.3)
        second, _ = pool.rate(0.3, level0=1)  # the same workers serve the next step
    finally:
        pool.close()
    assert first > 0 and second > 0 and longest > 0
    # two workers each run the one-core sample: the sum exceeds one worker's rate (loose
    # bounds: the host may be busy with other work)
    assert 0.5 * one < first < 6 * one
    assert all(not p.is_alive() for p in pool.procs)
    assert "2 spawned single-threaded processes" in bench.all_core_sample(pool.n, longest, 0.3)
