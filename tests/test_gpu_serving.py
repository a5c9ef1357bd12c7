"""Serving loop: continuous batching of trace jobs, HBM-budget admission, p50/p99.

Each job's result must be the same alone (a plain mlmc_level_trace call) and in
a mix of concurrently running jobs on different lattices; the kernels are
per-system and the reductions fixed-order, so equality is exact.
"""

import numpy as np
import pytest

import inputs

pkg = pytest.importorskip("paper_2212_04430_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as g
    g.build()


def _jobs():
    rng = np.random.default_rng(404)
    specs = []
    lattices = [(4, 4, 4, 4), (4, 4, 2, 8), (6, 4, 4, 4)]
    for k in range(7):
        dims = lattices[k % 3]
        nlev = 2 + k % 3
        sig = np.sort(np.exp(rng.uniform(np.log(0.005), 0.0, size=nlev)))
        specs.append(dict(dims=dims, gseed=5000 + k, m=-0.3, sigmas=sig, gamma=pkg.gamma_matrix(["g3", "g5g4", "1"][k % 3]),
                          p=k % 3, n=[int(rng.integers(4, 12))] * nlev, seed=6000 + k,
                          est=["diff", "split_even", "product"][k % 3], prec=["f16", "f32", "bf16"][k % 3]))
    return specs


def _run_alone(s, u):
    ctx = pkg.Context(s["dims"])
    ctx.fs_set_gauge(u)
    out = ctx.mlmc_level_trace(s["m"], s["sigmas"], s["gamma"], s["p"], s["n"], seed=s["seed"], job=1,
                               estimator=s["est"], prec=s["prec"], rhs_tile=8)
    ctx.close()
    return out


def test_jobs_identical_alone_and_in_a_concurrent_mix():
    specs = _jobs()
    gauges = [inputs.gauge_field(s["dims"], "smooth", seed=s["gseed"], eps=0.4) for s in specs]
    alone = [_run_alone(s, u) for s, u in zip(specs, gauges)]
    srv = pkg.Server(device=0, hbm_budget_bytes=8 << 30, max_active=3)
    tickets = [srv.submit(s["dims"], u, s["m"], s["sigmas"], s["gamma"], s["p"], s["n"], s["seed"], job=1,
                          estimator=s["est"], prec=s["prec"], rhs_tile=8) for s, u in zip(specs, gauges)]
    results = [srv.poll(t) for t in tickets]
    for a, r in zip(alone, results):
        assert r["status"] == 0
        assert np.array_equal(r["trace"], a["trace"])
        assert np.array_equal(r["var"], a["var"])
    st = srv.stats()
    assert st["completed"] == len(specs) and st["queued"] == 0 and st["active"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["reserved_bytes"] == 0
    srv.close()


def test_budget_admission_and_poll_timeout():
    dims = (8, 8, 8, 8)
    u = inputs.gauge_field(dims, "smooth", seed=77, eps=0.3)
    g = pkg.gamma_matrix("g5g3")
    # a budget that fits one such job at a time: jobs run one after another and all finish
    srv = pkg.Server(device=0, hbm_budget_bytes=150 << 20, max_active=4)
    tickets = [srv.submit(dims, u, -0.2, [0.02, 0.1, 0.5], g, 2, [16, 16, 16], seed=9 + k, prec="f32",
                          rhs_tile=16) for k in range(3)]
    first = srv.poll(tickets[-1], timeout_ms=0)  # the last job cannot be done yet
    assert first is None
    res = [srv.poll(t) for t in tickets]
    assert all(r["status"] == 0 for r in res)
    # FIFO under a one-job budget: each job waited for the previous ones
    assert res[2]["queue_ms"] >= res[1]["queue_ms"] >= res[0]["queue_ms"]
    # a job larger than the whole budget is refused at submission
    with pytest.raises(pkg.FsError) as e:
        srv.submit((16, 16, 16, 32), inputs.unit_gauge((16, 16, 16, 32)), -0.2, [0.1, 0.5], g, 1, [8, 8], seed=1,
                   prec="f32", rhs_tile=32)
    assert e.value.code == pkg.fsmlmc.FS_ERR_BUDGET
    with pytest.raises(pkg.FsError):
        srv.poll(123456789, timeout_ms=0)  # unknown ticket
    srv.close()


def test_probed_and_expanded_jobs_in_a_concurrent_mix():
    """Jobs with probing colours, spin-colour dilution and the hopping parameter expansion run
    concurrently with plain ones (every job copies its own colour table; every worker context
    uploads its own): each result equals the job run alone."""
    from oracle import probing as opr  # the colours are inputs here; the library does not use the oracle
    specs = []
    for k, dims in enumerate([(4, 4, 4, 4), (4, 4, 8, 4), (4, 4, 4, 8), (6, 4, 4, 4)]):
        col, nc = opr.greedy_coloring(dims, 1 + k % 2, k % 3)
        specs.append(dict(dims=dims, u=inputs.gauge_field(dims, "smooth", seed=7000 + k, eps=0.4),
                          sig=[0.05, 0.3 + 0.1 * k], n=[2, 3], p=k % 3, seed=8000 + k,
                          extra=[dict(colors=col, ncolors=nc, dilute=True), dict(hpe_order=4),
                                 dict(colors=col, ncolors=nc, hpe_order=2), {}][k]))
    g = pkg.gamma_matrix("g3")
    kw = dict(prec="f16", tol=1e-8, rhs_tile=16)
    alone = []
    for s in specs:
        ctx = pkg.Context(s["dims"])
        ctx.fs_set_gauge(s["u"])
        alone.append(ctx.mlmc_level_trace(-0.1, s["sig"], g, s["p"], s["n"], seed=s["seed"], lanes=1, **kw,
                                          **s["extra"]))
        ctx.close()
    srv = pkg.Server(device=0, hbm_budget_bytes=16 << 30, max_active=4)
    tickets = [srv.submit(s["dims"], s["u"], -0.1, s["sig"], g, s["p"], s["n"], s["seed"], **kw, **s["extra"])
               for s in specs]
    results = [srv.poll(t) for t in tickets]
    srv.close()
    for a, r in zip(alone, results):
        assert r["status"] == 0
        assert np.array_equal(r["trace"], a["trace"]) and np.array_equal(r["var"], a["var"])


def test_least_work_first_admission():
    """With one worker busy, a large and then a small job queue up: the small one starts first
    (least work first); with FIFO requested, the large one does; a job older than max_wait_ms goes
    next whatever its size."""
    small, large = (4, 4, 4, 4), (8, 8, 8, 8)
    u_s = inputs.gauge_field(small, "smooth", seed=91, eps=0.3)
    u_l = inputs.gauge_field(large, "smooth", seed=92, eps=0.3)
    g = pkg.gamma_matrix("g3")
    kw = dict(prec="f32", tol=1e-8, rhs_tile=16)

    def order(least_work_first, max_wait_ms):
        srv = pkg.Server(device=0, hbm_budget_bytes=8 << 30, max_active=1)
        srv.set_admission(least_work_first, max_wait_ms)
        busy = srv.submit(large, u_l, -0.2, [0.02, 0.3], g, 1, [48, 48], seed=1, **kw)  # occupies the worker
        big = srv.submit(large, u_l, -0.2, [0.02, 0.3], g, 1, [16, 16], seed=2, **kw)
        tiny = srv.submit(small, u_s, -0.2, [0.3], g, 0, [2], seed=3, **kw)
        r = {k: srv.poll(t) for k, t in (("busy", busy), ("big", big), ("tiny", tiny))}
        srv.close()
        assert all(x["status"] == 0 for x in r.values())
        return r

    r = order(True, 60000.0)
    assert r["tiny"]["queue_ms"] < r["big"]["queue_ms"]
    r = order(False, 60000.0)
    assert r["big"]["queue_ms"] < r["tiny"]["queue_ms"]
    r = order(True, 0.0)  # every queued job counts as waited out: oldest first
    assert r["big"]["queue_ms"] < r["tiny"]["queue_ms"]
