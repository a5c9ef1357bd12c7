"""bench.py's multi-GPU form on CPU: two gloo ranks (world size 2) run the replica
bookkeeping and the timing reductions the GPU run uses with NCCL.

Replicas only (the systems are independent): no data-path collective. The whole-job
rate is the solves of all ranks over the slowest rank's time, and replicas draw
disjoint noise job ids.
"""

import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_setup("gloo")
    assert (w, r, local) == (ws, rank, rank)
    bench.barrier(w)
    # rank r took (r + 1) * 10 ms for 224 * 3 solves
    rate, ms_max, total = bench.whole_job_rate(10.0 * (rank + 1), 224.0 * 3, w)
    jobs = [bench.job_base(rank) + off + k for off in (0, 1000, 2000) for k in range(999)]
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"rate": rate, "ms_max": ms_max, "total": total, "jobs": [min(jobs), max(jobs)]}, f)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    ws = 2
    mp.start_processes(_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(ws)]
    for r in res:
        assert r["ms_max"] == 20.0
        assert r["total"] == 224.0 * 3 * ws
        assert r["rate"] == pytest.approx(224.0 * 3 * ws / 0.020)
    # noise job ids of the two replicas (warm-up, timed, end to end) do not overlap
    (a0, a1), (b0, b1) = res[0]["jobs"], res[1]["jobs"]
    assert a1 < b0 or b1 < a0


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    rate, ms_max, total = bench.whole_job_rate(50.0, 100.0, 1)
    assert (rate, ms_max, total) == (2000.0, 50.0, 100.0)
