#!/usr/bin/env python3
"""Benchmark: Frequency-Splitting MLMC shifted Wilson solves per second on GB300.

One step = one mlmc_level_trace call (the whole hot path: Z4 noise on the
device, even-odd shifted solves at every level, Gamma Omega_p contraction,
per-level trace and practical variance) over `--vectors` noise vectors per
level. Default workload: 16^3x32 lattice, smoothed links U = exp(i 0.4 H),
m = -0.35, 4-level FS shifts {0.005, 0.03, 0.15, 0.6}, Gamma = gamma_3, p = 4,
32-system tiles, FP16 spinor storage with FP32 arithmetic, 12-real links, FP64
reliable updates, solves to FP64 relative residual 1e-8.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "shifted Wilson solves/s at 1e-8 resid; dslash HBM GB/s vs peak; p50/p99 latency"

WORKLOADS = {
    # the 16^3x32 FS-MLMC job (4 levels, 512 Z4 vectors per level in 32-system tiles); a step is a
    # quarter of it, 128 vectors per level (the tiles drain once per call: 32 per call lost 8%)
    "16x32": dict(key="16x32", dims=(16, 16, 16, 32), eps=0.4, gauge_seed=1003, noise_seed=2003, m=-0.35,
                  sigmas=[0.005, 0.03, 0.15, 0.6], gamma="g3", p=4, vectors=128, tile=32, prec="f16",
                  link=12, tol=1e-8, estimator="split_even",
                  name="16^3x32 Wilson FS-MLMC, 4 levels {0.005,0.03,0.15,0.6}, m=-0.35, eps=0.4, gamma3, p=4"),
    # the 8^4 FS-MLMC job (3 levels, 256 Z4 vectors per level in 16-system tiles)
    "8x8": dict(key="8x8", dims=(8, 8, 8, 8), eps=0.3, gauge_seed=1002, noise_seed=2002, m=-0.2,
                sigmas=[0.02, 0.1, 0.5], gamma="g5g3", p=2, vectors=256, tile=16, prec="f32", link=18,
                tol=1e-8, estimator="split_even",
                name="8^4 Wilson FS-MLMC, 3 levels {0.02,0.1,0.5}, m=-0.2, eps=0.3, gamma5 gamma3, p=2"),
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def hop_traffic_ratio(workload):
    """DRAM traffic / algorithmic bytes of the hop mix, from the committed ncu summary, if that
    summary was taken on the current kernel source (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "hop_kernel_%s.md" % workload)
    if not os.path.exists(path):
        return None
    src = b""
    for f in ("fs_hop.cuh", "fs_common.cuh", "fs_launch.cuh"):
        with open(os.path.join(ROOT, "paper_2212_04430_gb300", "csrc", f), "rb") as fh:
            src += fh.read()
    digest = hashlib.sha256(src).hexdigest()[:16]
    ratio, tag = None, None
    with open(path) as f:
        for line in f:
            if line.startswith("traffic_to_algorithmic_ratio:"):
                ratio = float(line.split(":")[1])
            if line.startswith("kernel_source_sha256_16:"):
                tag = line.split(":")[1].strip()
    return ratio if (tag == digest and ratio) else None


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs (clocks, throttle reasons, and the
    share of time a kernel of this GPU was running: the gaps the host's solve loops leave)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, busy, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
            if len(parts) > 9:
                try:
                    busy.append(float(parts[9]))
                except ValueError:
                    pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "gpu_busy_pct": statistics.mean(busy) if busy else None}


def measure_arith_peaks(pkg, index, seconds):
    """The FP32 and FP64 roofs measured on this GPU (fs_measure_peak: independent FMA chains on
    every SM), with the SM clock sampled while each runs; `at_max_clock` rescales the rate by
    max / median sampled clock (time x median MHz)."""
    out = {}
    for kind in ("f32", "f32x2", "f64"):
        clk = ClockSampler(index)
        clk.start()
        tf, ms = pkg.fs_measure_peak(kind, seconds)
        c = clk.stop()
        entry = {"tflops": tf, "ms": ms, "sm_mhz": c.get("sm_mhz"), "sm_max_mhz": c.get("sm_max_mhz"),
                 "reasons": c.get("reasons")}
        if c.get("sm_mhz") and c.get("sm_max_mhz"):
            entry["at_max_clock"] = tf * c["sm_max_mhz"] / c["sm_mhz"]
        out[kind] = entry
    out["how"] = ("fs_measure_peak: 8 independent multiply-add chains per thread, all SMs filled, "
                  "launches repeated for %.1f s, timed with CUDA events; 2 flop per multiply-add" % seconds)
    return out


def dist_setup(backend="nccl"):
    """Replicas only: one process per GPU, each solving its own noise vectors. The process
    group carries nothing but the barrier and the two scalar reductions of the timing."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
    return ws, rank, local


def _reduce_device():
    import torch.distributed as dist
    return "cpu" if dist.get_backend() == "gloo" else "cuda"


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_base(rank):
    """First noise job id of a replica: warm-up, timed and end-to-end steps use
    base + k, base + 1000 + k and base + 2000 + k, so replicas never share a Z4 vector."""
    return 100000 * rank


def whole_job_rate(ms_local, solves_local, ws):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    ms_max = max_over_ranks(ms_local, ws)
    total = sum_over_ranks(solves_local, ws)
    return total / (ms_max / 1e3), ms_max, total


# --------------------------------------------------------------------------- CPU oracle
def oracle_rate(w, budget_s, seed_level=0, sync=None):
    """Oracle solves/s: a bounded number of oracle BiCGStab iterations on one system of the
    workload, converted with the oracle's own iterations per solve (oracle/baseline_iters.json).
    `sync`, if given, is called between the setup and the timed work (the all-core leg lines
    its workers up there)."""
    from oracle import dirac, philox, solve
    import inputs
    dims = w["dims"]
    u = inputs.gauge_field(dims, "smooth", seed=w["gauge_seed"], eps=w["eps"])
    shp = dirac.lattice_shape(dims)
    ul = u.reshape((4,) + shp + (3, 3))
    v = int(np.prod(dims))
    lev = seed_level % len(w["sigmas"])
    sigma = w["sigmas"][lev]
    z = philox.z4_noise(v, w["noise_seed"], 0, lev, 0).ravel()

    def apply_A(vec):
        return dirac.apply_D(ul, vec.reshape(shp + (4, 3)), w["m"], sigma, -1).ravel()

    if sync is not None:
        sync()
    t = time.time()
    apply_A(z)
    t_apply = time.time() - t
    iters = max(1, int(budget_s / (2.0 * t_apply)))
    t = time.time()
    solve.bicgstab(apply_A, z, tol=1e-30, max_iter=iters)
    dt = time.time() - t - t_apply  # bicgstab also applies A once for the final true residual
    per_iter = dt / iters
    with open(os.path.join(ROOT, "oracle", "baseline_iters.json")) as f:
        cal = json.load(f)[w["key"]]
    sig = w["sigmas"]
    it = [cal["iters"][repr(s)] for s in sig]
    L = len(sig) - 1
    mix = [it[l] + it[l + 1] for l in range(L)] + [it[L]]  # DIFF: two solves per sample below L
    nsolve = 2 * L + 1
    mean_iters = sum(mix) / nsolve
    rate = 1.0 / (per_iter * mean_iters)
    sample = ("%d oracle BiCGStab iterations (%.1f s) on one %s system at sigma=%g; "
              "solves/s = 1 / (s per iteration x %.1f oracle iterations per solve, the workload's "
              "shift mix from oracle/baseline_iters.json)" % (iters, dt, "x".join(map(str, dims)), sigma,
                                                             mean_iters))
    return rate, sample, dt


def _oracle_worker(w, tasks, results, barrier):
    """One host core of the all-core oracle leg: runs oracle_rate on the system it is given,
    timed only once every worker has finished its setup."""
    while True:
        task = tasks.get()
        if task is None:
            return
        budget, level = task
        try:
            r, _, dt = oracle_rate(w, budget, level, sync=lambda: barrier.wait(timeout=900))
            results.put((r, dt))
        except Exception as ex:  # a broken barrier releases the others at once
            barrier.abort()
            results.put(("failed", repr(ex)))


class OraclePool:
    """Independent oracle systems on all host cores at once: one spawned process per core,
    each single-threaded, the oracle's arithmetic unchanged. Throughput = the sum of the
    workers' rates, each measured while all of them run."""

    THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")

    def __init__(self, w, n=None):
        import multiprocessing as mp
        self.n = n or len(os.sched_getaffinity(0))
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in self.THREAD_VARS}
        for k in self.THREAD_VARS:
            os.environ[k] = "1"
        try:
            self.barrier = ctx.Barrier(self.n)
            self.tasks = [ctx.Queue() for _ in range(self.n)]
            self.results = ctx.Queue()
            self.procs = [ctx.Process(target=_oracle_worker, args=(w, q, self.results, self.barrier),
                                      daemon=True) for q in self.tasks]
            for p in self.procs:
                p.start()
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def rate(self, budget_s, level0=0):
        """(aggregate solves/s, the longest worker's timed seconds)."""
        for i, q in enumerate(self.tasks):
            q.put((budget_s, level0 + i))
        got = [self.results.get(timeout=4 * budget_s + 900) for _ in range(self.n)]
        bad = [g[1] for g in got if g[0] == "failed"]
        if bad:
            raise RuntimeError("oracle worker failed: %s" % bad[0])
        return float(sum(g[0] for g in got)), float(max(g[1] for g in got))

    def close(self):
        for q in self.tasks:
            q.put(None)
        for p in self.procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()


def all_core_sample(n, dt, budget_s):
    return ("%d spawned single-threaded processes (one per host core), each running the one-core "
            "sample on its own system (levels taken in turn) for about %.0f s (longest %.1f s) after "
            "a common barrier; solves/s = the sum of their rates" % (n, budget_s, dt))


def run_reference(args, w):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if int(os.environ.get("RANK", "0")) != 0:
        return  # the CPU oracle runs once, on rank 0
    budget = args.ref_budget
    pool = OraclePool(w)
    try:
        for k in range(args.warmup):
            pool.rate(min(budget, 3.0), k)
        rates = []
        t0 = time.time()
        for k in range(args.steps):
            r, dt = pool.rate(budget, k)
            rates.append(r)
        wall = time.time() - t0
    finally:
        pool.close()
    value = float(np.mean(rates))
    sample = all_core_sample(pool.n, dt, budget)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args, w),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": pool.n, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(args, w):
    return {"workload": w["name"], "lattice": "x".join(map(str, w["dims"])), "levels": len(w["sigmas"]),
            "vectors_per_level_per_step": args.vectors or w["vectors"], "estimator": w["estimator"],
            "rhs_tile": args.tile or w["tile"], "storage": w["prec"], "links": "%d-real" % w["link"],
            "tol": w["tol"], "delta": args.delta or "library", "lanes": args.lanes or "library",
            "l2": "working set above L2 (no flush needed)",
            "operator": "Wilson-clover, c_sw = %g" % args.clover if args.clover else "Wilson"}


# --------------------------------------------------------------------------- serving
SERVE_LATTICES = [(8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32)]
CLIFFORD = ["1", "g1", "g2", "g3", "g4", "g5", "g1g2", "g1g3", "g1g4", "g2g3", "g2g4", "g3g4", "g5g1", "g5g2",
            "g5g3", "g5g4"]


def run_serving(pkg, inputs, device, n_jobs, rate=20.0, budget_gb=60, max_active=4, seed=4004, vectors=(32, 256)):
    """Poisson arrivals (mean `rate` jobs/s) of trace jobs: lattice uniform over 8^4, 12^3x24,
    16^3x32; 2..6 log-uniform shifts in [0.005, 1]; `vectors` (32..256 in the serving workload)
    Z4 vectors per level; p in 0..4; Gamma uniform over the 16 Clifford products; FP16 or BF16
    inner solves; m = -0.2, eps = 0.3. One gauge field per lattice, shared by its jobs."""
    rng = np.random.default_rng(seed)
    gauges = {d: inputs.gauge_field(d, "smooth", seed=4100 + i, eps=0.3) for i, d in enumerate(SERVE_LATTICES)}
    jobs = []
    for k in range(n_jobs):
        dims = SERVE_LATTICES[int(rng.integers(len(SERVE_LATTICES)))]
        nlev = int(rng.integers(2, 7))
        sig = np.sort(np.exp(rng.uniform(np.log(0.005), 0.0, size=nlev)))
        jobs.append(dict(dims=dims, sig=sig, n=[int(rng.integers(vectors[0], vectors[1] + 1))] * nlev,
                         p=int(rng.integers(0, 5)),
                         gamma=pkg.gamma_matrix(CLIFFORD[int(rng.integers(16))]),
                         prec=["f16", "bf16"][int(rng.integers(2))], gap=float(rng.exponential(1.0 / rate))))
    srv = pkg.Server(device=device, hbm_budget_bytes=int(budget_gb) << 30, max_active=max_active)
    t0 = time.time()
    tickets = []
    t_next = t0
    for k, j in enumerate(jobs):
        t_next += j["gap"]
        dt = t_next - time.time()
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(j["dims"], gauges[j["dims"]], -0.2, j["sig"], j["gamma"], j["p"], j["n"],
                                  seed=7000 + k, job=k, prec=j["prec"], tol=1e-8, rhs_tile=32))
    res = [srv.poll(t) for t in tickets]
    wall = time.time() - t0
    st = srv.stats()
    srv.close()
    bad = [dict(status=r["status"], prec=j["prec"], lattice="x".join(map(str, j["dims"])),
                sigma_min=float(j["sig"][0]), noconv=r["noconv"], restarts=r["restarts"], max_iters=r["max_iters"])
           for r, j in zip(res, jobs) if r["status"] != 0]
    qms = np.array([r["queue_ms"] for r in res])
    svc = np.array([r["latency_ms"] - r["queue_ms"] for r in res])
    return {"jobs": n_jobs, "completed": int(st["completed"]), "arrival_rate_per_s": rate,
            "vectors_per_level": list(vectors), "budget_gb": budget_gb, "max_active": max_active,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"], "mean_ms": st["mean_ms"],
            "queue_ms_p50": float(np.percentile(qms, 50)), "queue_ms_p99": float(np.percentile(qms, 99)),
            "service_ms_p50": float(np.percentile(svc, 50)), "service_ms_p99": float(np.percentile(svc, 99)),
            "solves": int(st["solves"]), "solves_per_s": st["solves"] / wall, "wall_s": wall,
            "offered_solves_per_s": float(st["solves"]) / max(sum(j["gap"] for j in jobs), 1e-9),
            "gauge_reuses": int(st["gauge_reuses"]),
            "failed_jobs": len(bad), "failures": bad,
            "restarts": int(sum(r["restarts"] for r in res)), "max_iters": int(max(r["max_iters"] for r in res))}


# --------------------------------------------------------------------------- estimator choice
def run_estimators(pkg, ctx, w, kw, n=64, seed=9500):
    """The three level estimators of the telescoping sum on the workload, the same N_l each:
    per level the practical variance V_l (Eq. (practical_variance)), the solver cost C_l of one
    sample (the iterations of its solves: two for l < L, one for the last level) and V_l C_l, and
    the multilevel cost F^2 = (sum_l sqrt(V_l C_l))^2 of Eq. (ml_cost_shifts) (the cost of reaching
    a given variance, up to the factor 1/eps^2). The smallest F^2 is the cheapest estimator."""
    gam = pkg.gamma_matrix(w["gamma"])
    nl = len(w["sigmas"])
    res = {}
    for est in ("diff", "split_even", "product"):
        t0 = time.time()
        out = ctx.mlmc_level_trace(w["m"], w["sigmas"], gam, w["p"], [n] * nl, seed=seed, job=50,
                                   estimator=est, **kw)
        dt = time.time() - t0
        st = out["stats"]
        k, levels, F = 0, [], 0.0
        for lev in range(nl):
            per = 2 if lev < nl - 1 else 1
            its = [sum(st[k + s * per + q]["iters"] for q in range(per)) for s in range(n)]
            k += n * per
            c = float(np.mean(its))
            v = float(out["var"][lev])
            levels.append({"V": v, "C_iters": c, "VC": v * c,
                           "trace": [float(out["trace"][lev].real), float(out["trace"][lev].imag)]})
            F += np.sqrt(max(v, 0.0) * c)
        res[est] = {"levels": levels, "F2": float(F * F), "V_FS_at_N": float(out["v_fs"]),
                    "total": [float(out["total"].real), float(out["total"].imag)], "seconds": dt,
                    "solves": int(len(st))}
    best = min(res, key=lambda e: res[e]["F2"])
    res["cheapest"] = best
    res["note"] = ("%d Z4 vectors per level, the same noise for every estimator (seed %d); F2 = "
                   "(sum_l sqrt(V_l C_l))^2 with C_l in BiCGStab iterations per sample" % (n, seed))
    return res


def run_clover(pkg, ctx, w, kw, n=64, c_sw=1.0, seed=9600):
    """The same level traces with the Wilson and the Wilson-clover operator (Sec. 4 computes with
    the clover discretisation), n Z4 vectors per level, one timed step each on the same noise:
    solves/s, BiCGStab iterations, and the cost of one system-iteration (the clover M-hat adds
    two site-local passes per application: (A + C_oo)^-1 on H_oe p and C_ee p)."""
    import torch
    gam = pkg.gamma_matrix(w["gamma"])
    nl = len(w["sigmas"])
    res = {}
    stream = torch.cuda.current_stream()
    for name, c in (("wilson", 0.0), ("clover", c_sw)):
        t0 = time.time()
        ctx.fs_set_clover(c)
        build_s = time.time() - t0
        ctx.mlmc_level_trace(w["m"], w["sigmas"], gam, w["p"], [4] * nl, seed=seed, job=60, estimator=w["estimator"],
                             **kw)  # warm-up: graphs and clover fields of this tile
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = ctx.mlmc_level_trace(w["m"], w["sigmas"], gam, w["p"], [n] * nl, seed=seed, job=61,
                                   estimator=w["estimator"], **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        if out["rc"] != 0:
            raise RuntimeError("%s solves did not converge: %s" % (name, ctx.last_error()))
        s = e0.elapsed_time(e1) / 1e3
        its = [st["iters"] for st in out["stats"]]
        res[name] = {"solves_per_s": len(its) / s, "seconds": s, "solves": len(its),
                     "mean_iters": float(np.mean(its)), "system_iterations_per_s": float(np.sum(its)) / s,
                     "max_true_resid": float(max(st["true_resid"] for st in out["stats"])),
                     "total": [float(out["total"].real), float(out["total"].imag)]}
        if c:
            res[name]["c_sw"] = c
            res[name]["table_build_s"] = build_s
            if w["m"] + w["sigmas"][-1] > 0:
                # the generalised hopping parameter expansion of the last level (Sec. 3.1)
                res[name]["hpe"] = run_hpe(pkg, ctx, w, kw)
    ctx.fs_set_clover(0.0)
    res["iteration_cost_ratio"] = res["wilson"]["system_iterations_per_s"] / res["clover"]["system_iterations_per_s"]
    res["note"] = ("%d Z4 vectors per level (seed %d), the workload's precision, tile and lanes; "
                   "iteration_cost_ratio = Wilson / clover system-iterations per second" % (n, seed))
    return res


# --------------------------------------------------------------------------- the full method
def run_pipeline(pkg, ctx, w, kw, levels=4, n_s=5, n_ref=512, n_max=128, seed=9000, hpe_order=0):
    """The paper's procedure end to end on the workload's lattice: variance sampling at the
    sampling shifts (Sec. 3.1, N_s = 5 as in the paper), interpolation and optimal shifts
    (Sec. 3.2-3.3), sample allocation for a target variance (Eq. (num_samples)), then the
    split-even level traces (Eq. (fs_trace_est)) whose variance the sampling predicts.
    Target: the variance of a single-level estimator at sigma_0 with n_ref vectors. N_l is
    capped at n_max to bound the run; the measured V_l are compared with the predictions.
    hpe_order = K follows the paper further: V_L is sampled with the hopping parameter expansion
    at the sampling shifts with m + s > 0, and the last level uses it when m + sigma_L > 0."""
    s_hat = [w["sigmas"][0], 0.05, 0.25, 0.5, 1.0]  # sigma_0 = the workload's first shift
    gam = pkg.gamma_matrix(w["gamma"])
    t0 = time.time()
    vs = ctx.variance_sample(w["m"], s_hat, gam, [w["p"]], n_s, seed=seed, job=1, hpe_order=hpe_order, **kw)
    t_vs = time.time() - t0
    s = pkg.fs_eval_grid(s_hat)
    t1 = time.perf_counter()
    sel = pkg.fs_select_shifts(s_hat, vs["VL"][0], vs["Vbar"][0], vs["iters"], s, levels - 1)
    t_sel = time.perf_counter() - t1
    eps2 = vs["VL"][0][0] / n_ref
    N, mu, v_fs, c_fs = pkg.fs_sample_allocation(sel["V"], sel["C"], eps2)
    n_use = [int(min(max(1, np.ceil(x)), n_max)) for x in N]
    t2 = time.time()
    out = ctx.mlmc_level_trace(w["m"], sel["sigma"], gam, w["p"], n_use, seed=seed, job=2, estimator="split_even",
                               hpe_order=hpe_order, **kw)
    t_tr = time.time() - t2
    var_meas = [float(v) for v in out["var"]]
    import math
    return {"hpe_order": hpe_order, "sampling_shifts": s_hat, "n_s": n_s, "evaluation_shifts": len(s),
            "levels": levels,
            "sigma": [float(x) for x in sel["sigma"]],
            "V_pred": [float(x) for x in sel["V"]], "V_meas": var_meas,
            "iters_sampled": [float(x) for x in vs["iters"]], "C_pred": [float(x) for x in sel["C"]],
            "eps2": eps2, "N_opt": [float(x) for x in N], "N_used": n_use,
            "V_FS_pred_at_N_used": float(sum(v / n for v, n in zip(sel["V"], n_use))),
            "V_FS_meas_at_N_used": float(sum(v / n for v, n in zip(var_meas, n_use))),
            "cost_ratio_pred": float(c_fs / (n_ref * vs["iters"][0])),
            "brute_force_combinations": math.comb(len(s) - 1, levels - 1),
            "t_variance_sample_s": t_vs, "t_select_ms": 1e3 * t_sel, "t_level_traces_s": t_tr,
            "solves": int(len(out["stats"])), "rc": int(out["rc"])}


def run_probing(pkg, ctx, w, kw, p=4, k=4, n_s=1, seed=9100):
    """Probed and spin-colour diluted level traces on the workload's lattice (Sec. 2.1, Sec. 3.1):
    displacement-p distance-k colours (the paper's p4k4 set; the greedy colouring of the library)
    and full dilution, n_s samples per level, each the sum over its 12 c pieces. The pieces are
    sparse right-hand sides generated on the device; solves/s is timed with CUDA events."""
    import torch
    t0 = time.perf_counter()
    col, nc = pkg.fs_probing_colors(w["dims"], k, p)
    t_col = time.perf_counter() - t0
    gam = pkg.gamma_matrix(w["gamma"])
    n = [n_s] * len(w["sigmas"])
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = ctx.mlmc_level_trace(w["m"], w["sigmas"], gam, w["p"], n, seed=seed, job=1, estimator=w["estimator"],
                               colors=col, ncolors=nc, dilute=True, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    if out["rc"] != 0:
        raise RuntimeError("probed solves did not converge: %s" % ctx.last_error())
    solves = len(out["stats"])
    sec = e0.elapsed_time(e1) / 1e3
    return {"value": solves / sec, "unit": "solves/s", "probing": "p%dk%d" % (p, k), "colors": int(nc),
            "pieces_per_sample": 12 * int(nc), "samples_per_level": n_s, "solves": solves, "seconds": sec,
            "t_coloring_s": t_col, "mean_iters": float(np.mean([st["iters"] for st in out["stats"]])),
            "trace": [[float(t.real), float(t.imag)] for t in out["trace"]]}


def run_hpe(pkg, ctx, w, kw, K=4, n=64, seed=9200):
    """The last level of the workload with and without the hopping parameter expansion to order K
    (Sec. 3.1; the last shift has m + sigma_L > 0): the exact low orders from displacement-p
    distance-(K-1) probing, n Z4 samples of each estimator, their variances and times."""
    import torch
    sig = [w["sigmas"][-1]]
    gam = pkg.gamma_matrix(w["gamma"])
    stream = torch.cuda.current_stream()
    res = {}
    for name, order in (("plain", 0), ("hpe", K)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = ctx.mlmc_level_trace(w["m"], sig, gam, w["p"], [n], seed=seed, job=1, hpe_order=order, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        if out["rc"] != 0:
            raise RuntimeError("last-level solves did not converge: %s" % ctx.last_error())
        res[name] = (out, e0.elapsed_time(e1) / 1e3)
    (po, pt), (ho, ht) = res["plain"], res["hpe"]
    return {"order": K, "sigma_L": sig[0], "m_plus_sigma_L": w["m"] + sig[0], "samples": n,
            "var_plain": float(po["var"][0]), "var_hpe": float(ho["var"][0]),
            "variance_ratio": float(po["var"][0] / ho["var"][0]) if ho["var"][0] > 0 else None,
            "trace_plain": [float(po["trace"][0].real), float(po["trace"][0].imag)],
            "trace_hpe": [float(ho["trace"][0].real), float(ho["trace"][0].imag)],
            "seconds_plain": pt, "seconds_hpe": ht,
            "note": "seconds_hpe includes the exact low orders (12 c probing vectors, K-1 FP64 kappa H each)"}


def run_variance_24x64(pkg, inputs, device, n_s=24, seed=2005):
    """The 24^3x64 variance-sampling job (5 sampling shifts, p = 0..8, FP16 storage, 12-real links,
    64-system tiles, groups of 10 systems per noise vector refilled as slots free) on n_s Z4 vectors: solves/s through variance_sample, timed
    with CUDA events; the gauge upload is outside the timed region."""
    import torch
    dims = (24, 24, 24, 64)
    u = inputs.gauge_field(dims, "smooth", seed=1005, eps=0.5)
    ctx = pkg.Context(dims, bc_t=-1, device=device)
    stream = torch.cuda.current_stream()
    try:
        ctx.set_stream(stream.cuda_stream)
        ctx.fs_set_gauge(u)
        s_hat = [0.0, 0.05, 0.25, 0.5, 1.0]
        kw = dict(prec="f16", tol=1e-8, rhs_tile=64, link_compress=12)
        g = pkg.gamma_matrix("g3")
        ctx.variance_sample(-0.38, s_hat, g, list(range(9)), 1, seed=seed, job=0, **kw)  # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = ctx.variance_sample(-0.38, s_hat, g, list(range(9)), n_s, seed=seed, job=1, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        if out["rc"] != 0:
            raise RuntimeError("24^3x64 solves did not converge: %s" % ctx.last_error())
        sec = e0.elapsed_time(e1) / 1e3
        solves = 2 * len(s_hat) * n_s
        return {"workload": "24^3x64 variance sampling, eps=0.5, m=-0.38, s_hat={0,0.05,0.25,0.5,1.0}, gamma3, "
                            "p=0..8, FP16 storage, 12-real links, 64-system tiles",
                "value": solves / sec, "unit": "solves/s", "solves": solves, "seconds": sec,
                "mean_iters_per_shift": [float(x) for x in out["iters"]],
                "device_bytes": int(ctx.device_bytes())}
    finally:
        ctx.close()


def run_pipeline_paper_noise(pkg, ctx, w, kw, levels=4, n_s=5, n_max=4, seed=9300):
    """The paper's procedure with the paper's noise (Sec. 4: 5 Z4 vectors, full spin-colour
    dilution, p8k7 probing colours; Sec. 3.1: the hopping parameter expansion of order 4 where
    m + s > 0): variance sampling, shift selection, sample allocation for a target variance
    (a twentieth of the sampled single-level variance at sigma_0), then the split-even level
    traces with the same noise, N_l capped at n_max probed samples."""
    import math
    s_hat = [w["sigmas"][0], 0.05, 0.25, 0.5, 1.0]
    gam = pkg.gamma_matrix(w["gamma"])
    t0 = time.perf_counter()
    col, nc = pkg.fs_probing_colors(w["dims"], 7, 8)
    t_col = time.perf_counter() - t0
    noise = dict(colors=col, ncolors=nc, dilute=True, hpe_order=4)
    t0 = time.time()
    vs = ctx.variance_sample(w["m"], s_hat, gam, [w["p"]], n_s, seed=seed, job=1, **noise, **kw)
    t_vs = time.time() - t0
    s = pkg.fs_eval_grid(s_hat)
    sel = pkg.fs_select_shifts(s_hat, vs["VL"][0], vs["Vbar"][0], vs["iters"], s, levels - 1)
    eps2 = vs["VL"][0][0] / 20.0
    N, mu, v_fs, c_fs = pkg.fs_sample_allocation(sel["V"], sel["C"], eps2)
    n_use = [int(min(max(1, math.ceil(x)), n_max)) for x in N]
    t2 = time.time()
    out = ctx.mlmc_level_trace(w["m"], sel["sigma"], gam, w["p"], n_use, seed=seed, job=2, estimator="split_even",
                               **noise, **kw)
    t_tr = time.time() - t2
    return {"probing": "p8k7", "colors": int(nc), "t_coloring_s": t_col, "dilution": "full spin-colour",
            "hpe_order": 4, "n_s": n_s, "sampling_shifts": s_hat,
            "variance_sample_solves": 12 * int(nc) * len(s_hat) * n_s, "t_variance_sample_s": t_vs,
            "VL_sampled": [float(x) for x in vs["VL"][0]], "sigma": [float(x) for x in sel["sigma"]],
            "V_pred": [float(x) for x in sel["V"]], "N_opt": [float(x) for x in N], "N_used": n_use,
            "V_meas": [float(v) for v in out["var"]], "trace_levels": [[float(t.real), float(t.imag)]
                                                                       for t in out["trace"]],
            "level_trace_solves": int(len(out["stats"])), "t_level_traces_s": t_tr, "rc": int(out["rc"])}


# --------------------------------------------------------------------------- GPU arm
def build_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="16x32", choices=sorted(WORKLOADS))
    ap.add_argument("--vectors", type=int, default=0, help="Z4 vectors per level per step")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--delta", type=float, default=0.0,
                    help="reliable-update trigger factor (0: library choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lanes", type=int, default=0, help="tiles solved at once (0: library choice)")
    ap.add_argument("--no-fp64-baseline", action="store_true", help="skip the FP64 single-RHS GPU solver")
    ap.add_argument("--roof-steps", type=int, default=2, help="single-lane steps timed for the roofline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-peaks", action="store_true", help="skip the measured FP32 / FP64 roofs")
    ap.add_argument("--no-estimators", action="store_true", help="skip the DIFF / SPLIT_EVEN / PRODUCT comparison")
    ap.add_argument("--peak-seconds", type=float, default=2.0, help="timed seconds per measured roof")
    ap.add_argument("--ref-budget", type=float, default=8.0, help="seconds of oracle work per reference step")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--serve-jobs", type=int, default=200, help="jobs in the 20 jobs/s serving run (0: skip)")
    ap.add_argument("--stable-jobs", type=int, default=200, help="jobs in the stable-load serving run (0: skip)")
    ap.add_argument("--stable-rate", type=float, default=4.0, help="arrival rate of the stable-load run, jobs/s")
    ap.add_argument("--no-large", action="store_true", help="skip the 24^3x64 variance-sampling measurement")
    ap.add_argument("--no-probing", action="store_true",
                    help="skip the probed and spin-colour diluted level traces (p4k4 colours)")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="skip the end-to-end run of variance sampling, shift selection and allocation")
    ap.add_argument("--clover", type=float, default=0.0,
                    help="c_sw of the Wilson-clover operator for the whole timed step (0: Wilson)")
    ap.add_argument("--no-clover", action="store_true", help="skip the Wilson / Wilson-clover comparison")
    return ap


def main():
    ap = build_parser()
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    if args.warmup < 1:
        ap.error("--warmup must be >= 1")
    if args.steps >= 1000 or args.warmup >= 1000:
        ap.error("--steps and --warmup must be below 1000 (noise job ids of a replica)")

    ws, rank, local = dist_setup()
    import torch

    import inputs
    import paper_2212_04430_gb300 as pkg

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()  # a dedicated stream: the library launches on it, the events time it
    torch.cuda.set_stream(stream)
    dims = w["dims"]
    nvec = args.vectors or w["vectors"]
    tile = args.tile or w["tile"]
    u = inputs.gauge_field(dims, "smooth", seed=w["gauge_seed"], eps=w["eps"])
    ctx = pkg.Context(dims, bc_t=-1, device=local)
    ctx.set_stream(stream.cuda_stream)
    ctx.fs_set_gauge(u)
    if args.clover:
        ctx.fs_set_clover(args.clover)  # the table is rebuilt by every fs_set_gauge below
    gam = pkg.gamma_matrix(w["gamma"])
    kw = dict(prec=w["prec"], tol=w["tol"], rhs_tile=tile, link_compress=w["link"], delta=args.delta)
    n = [nvec] * len(w["sigmas"])

    def step(job, lanes=None):
        out = ctx.mlmc_level_trace(w["m"], w["sigmas"], gam, w["p"], n, seed=w["noise_seed"],
                                   job=job, estimator=w["estimator"],
                                   lanes=args.lanes if lanes is None else lanes, **kw)
        if out["rc"] != 0:
            raise RuntimeError("solver did not converge: %s" % ctx.last_error())
        return out

    solves_per_step = 2 * nvec * (len(w["sigmas"]) - 1) + nvec
    job0 = job_base(rank)
    for k in range(args.warmup):
        step(job0 + k)
    torch.cuda.synchronize()

    # ---- device-resident timed region (the library's own launch shape: three lanes by default)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    l0 = pkg.fsmlmc.fs_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters, updates, restarts, resid = [], [], [], []
    for k in range(args.steps):
        out = step(job0 + 1000 + k)
        iters.extend(s["iters"] for s in out["stats"])
        updates.extend(s["reliable_updates"] for s in out["stats"])
        restarts.extend(s["restarts"] for s in out["stats"])
        resid.extend(s["true_resid"] for s in out["stats"])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    launches = pkg.fsmlmc.fs_kernel_launches() - l0
    clk = clocks.stop()
    value, ms_max, total_solves = whole_job_rate(ms, solves_per_step * args.steps, ws)

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        upin = torch.empty(u.size * 2, dtype=torch.float64, pin_memory=True)
        upin.numpy()[:] = u.view(np.float64).ravel()
        h2d = upin.numel() * 8
        d2h = (len(n) * 2 + len(n) + sum(n) * 2) * 8
        barrier(ws)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for k in range(args.steps):
            ctx.fs_set_gauge(upin.numpy())
            step(job0 + 2000 + k)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(f0.elapsed_time(f1), ws)
        e2e = {"value": total_solves / (e2e_ms / 1e3), "unit": "solves/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # ---- one lane, no profiling: how much of the time a kernel runs while the host's solve loop
    # checks the tiles every few iterations (the headline's three lanes hide these gaps)
    single = None
    if rank == 0:
        s_clk = ClockSampler(torch.cuda.current_device())
        s_clk.start()
        torch.cuda.synchronize()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        step(job0 + 5000, lanes=1)
        h1.record(stream)
        torch.cuda.synchronize()
        sc = s_clk.stop()
        single = {"solves_per_s": solves_per_step / (h0.elapsed_time(h1) / 1e3), "gpu_busy_pct": sc.get("gpu_busy_pct"),
                  "samples": sc.get("samples"),
                  "note": "one step on one lane; gpu_busy_pct = nvidia-smi utilization.gpu, the share of time a "
                          "kernel was running, averaged over the samples"}

    # ---- roofline pass: the same step on one lane, every hop launch timed with CUDA events on
    # its stream (with several lanes a launch shares the GPU with the other lanes' kernels, and its
    # duration would measure that sharing rather than the kernel)
    ctx.profile_enable(True)
    for k in range(args.roof_steps):
        step(job0 + 3000 + k, lanes=1)
    prof = ctx.profile_read()
    prof64 = ctx.profile_read_fp64()
    ctx.profile_enable(False)

    # ---- the FP32 and FP64 roofs of this GPU, measured (rank 0; the GPU is otherwise idle here)
    arith = None
    if rank == 0 and not args.no_peaks:
        arith = measure_arith_peaks(pkg, torch.cuda.current_device(), args.peak_seconds)

    peaks, peak_kind = load_peaks()
    roof = None
    if prof["launches"] > 0 and prof["ms"] > 0:
        per_launch_s = prof["ms"] / prof["launches"] / 1e3
        bytes_per_launch = prof["bytes"] / prof["launches"]
        achieved = bytes_per_launch / per_launch_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "kernel": "hop_kernel (even-odd Wilson hopping term, inner precision)",
                "launches": prof["launches"], "avg_launch_us": per_launch_s * 1e6,
                "algorithmic_bytes_per_launch": bytes_per_launch, "peak_source": peak_kind,
                "pass": "hop launches of %d single-lane steps of the same workload, timed with CUDA events on "
                        "their stream" % args.roof_steps}
        ratio = hop_traffic_ratio(args.workload)
        if ratio is not None:
            roof["traffic"] = ratio * bytes_per_launch
        # the second roof of the same kernel: FP32 arithmetic, 1320 flop per (site, system) (at 32
        # systems and FP16 storage the kernel's 12.9 flop/B sits on the ridge of the two roofs),
        # against the FP32 rate measured on this GPU (else the nominal unit count x max clock)
        alu = 1320.0 * prof["site_systems"] / prof["launches"] / per_launch_s / 1e12
        if arith is not None:
            alu_peak = max(arith["f32"]["tflops"], arith["f32x2"]["tflops"])
            src = "measured (fs_measure_peak, the faster of scalar and packed FP32 FMA chains)"
        else:
            alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
            src = "nominal FP32 unit count x max clock"
        roof["second_roof"] = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "TFLOP/s",
                               "frac": alu / alu_peak, "peak_source": src}
        # the FP64-arithmetic work-list hops of the same pass (preparation, FP64 reliable-update
        # residuals, reconstruction, verification) against the measured FP64 rate
        if prof64["launches"] > 0 and prof64["ms"] > 0 and arith is not None:
            f64 = 1320.0 * prof64["site_systems"] / (prof64["ms"] / 1e3) / 1e12
            roof["fp64_hops"] = {"bound": "fp64", "achieved": f64, "peak": arith["f64"]["tflops"],
                                 "unit": "TFLOP/s", "frac": f64 / arith["f64"]["tflops"],
                                 "launches": prof64["launches"], "avg_launch_us": prof64["ms"] * 1e3 / prof64["launches"],
                                 "site_systems_per_launch": prof64["site_systems"] / prof64["launches"],
                                 "peak_source": "measured (fs_measure_peak, FP64 FMA chains)"}

    # ---- the plain FP64 single-RHS GPU solver (the same library in FP64 with one system per tile
    # and one lane: no reduced-precision storage, no batching) on a sample of the same job
    fp64 = None
    if not args.no_fp64_baseline and rank == 0:
        nb = max(1, nvec // 8)
        n64 = [nb] * len(w["sigmas"])
        solves64 = 2 * nb * (len(w["sigmas"]) - 1) + nb
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        out64 = ctx.mlmc_level_trace(w["m"], w["sigmas"], gam, w["p"], n64, seed=w["noise_seed"],
                                     job=job0 + 4000, estimator=w["estimator"], prec="f64", tol=w["tol"],
                                     rhs_tile=1, link_compress=18, lanes=1)
        g1.record(stream)
        torch.cuda.synchronize()
        if out64["rc"] != 0:
            raise RuntimeError("FP64 solver did not converge: %s" % ctx.last_error())
        v64 = solves64 / (g0.elapsed_time(g1) / 1e3)
        fp64 = {"value": v64, "unit": "solves/s", "value_over_this": value / v64,
                "sample": "%d Z4 vectors per level (%d solves) of the same job, FP64 storage and arithmetic, "
                          "one system per tile, one lane, tol %g" % (nb, solves64, w["tol"]),
                "mean_iters": float(np.mean([st["iters"] for st in out64["stats"]]))}

    pipeline = None
    if not args.no_pipeline and rank == 0:
        pipeline = run_pipeline(pkg, ctx, w, kw)
        # the paper's variant: V_L sampled with the hopping parameter expansion (order 4) where m + s > 0
        if not args.clover:  # the expansion is the Wilson operator's
            pipeline["with_hpe"] = run_pipeline(pkg, ctx, w, kw, hpe_order=4)
        # and with the paper's noise as well; an auxiliary measurement, so a failure is reported in
        # the line instead of ending the run
        try:
            pipeline["paper_noise"] = run_pipeline_paper_noise(pkg, ctx, w, kw)
        except Exception as ex:
            pipeline["paper_noise"] = {"error": str(ex)}

    estimators = None
    if not args.no_estimators and rank == 0:
        estimators = run_estimators(pkg, ctx, w, kw)

    clover = None
    if not args.no_clover and not args.clover and rank == 0:
        clover = run_clover(pkg, ctx, w, kw)

    large = None
    if not args.no_large and rank == 0:
        large = run_variance_24x64(pkg, inputs, local)

    probing = None
    if not args.no_probing and rank == 0:
        probing = run_probing(pkg, ctx, w, kw)
        if w["m"] + w["sigmas"][-1] > 0 and not args.clover:
            probing["hpe"] = run_hpe(pkg, ctx, w, kw)

    serving = serving_stable = None
    if args.serve_jobs > 0:
        # the serving workload at its arrival rate (20 jobs/s), above what one GPU serves: latency
        # there is mostly queueing
        serving = run_serving(pkg, inputs, local, args.serve_jobs)
    if args.stable_jobs > 0:
        # a stable queue: the same lattices, shifts, Gamma, p and precisions with 8..32 vectors per
        # level, arriving below the server's capacity, so latency is the batching's own
        serving_stable = run_serving(pkg, inputs, local, args.stable_jobs, rate=args.stable_rate, seed=4005,
                                     vectors=(8, 32))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            rate1, sample1, _ = oracle_rate(w, args.cpu_budget)
            one = {"value": rate1, "cores": 1, "sample": sample1}
            pool = OraclePool(w)
            try:
                rate, dt = pool.rate(args.cpu_budget)
            finally:
                pool.close()
            cpu = {"value": rate, "unit": "solves/s", "cores": pool.n, "kind": "oracle",
                   "sample": all_core_sample(pool.n, dt, args.cpu_budget), "one_core": one}
        except Exception as ex:  # the baseline never blocks the GPU line
            cpu = {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": "failed: %s" % ex}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_of(args, w), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "arith_peaks": arith, "serving": serving,
                "serving_stable": serving_stable, "estimators": estimators, "wilson_clover": clover,
                "single_lane": single,
                "pipeline": pipeline,
                "fp64_single_rhs": fp64, "probing": probing, "variance_sampling_24x64": large,
                "solver": {"mean_iters": float(np.mean(iters)) if iters else None,
                           "max_iters": int(max(iters)) if iters else None,
                           "mean_reliable_updates": float(np.mean(updates)) if updates else None,
                           "restarts": int(sum(restarts)),
                           "max_true_resid": float(max(resid)) if resid else None,
                           "true_resid_note": "the library's FP64 ||bhat - M x|| / ||z|| at the last reliable "
                                              "update of each timed solve (stopping rule: <= tol)",
                           "solves_per_step": solves_per_step}}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
