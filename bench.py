#!/usr/bin/env python
"""Benchmark of the exact isolated-value Mertens computation on GB300.

One step = one whole pass of the method for the workload (sieve of every block,
prefix scan, array update, resolve) -- mertens_run on a resident plan.  The
headline workload is a single query n = 10^16 with u = 4*10^10 and sieve
blocks of 2^28 y (the paper's Table 1 value M(10^16) = -3195437 is checked).

Prints ONE JSON line (rank 0).  Run `python bench.py --help` for options.
With --impl reference it times the plain CPU oracle instead, on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "update terms/s and wall time for M(10^16), M(10^18); batched-query p50/p99"
CONFIGS = {
    "1e16": dict(n=[10**16], u=4 * 10**10, block_len=1 << 28, pin=-3195437,
                 workload="single query n=1e16, u=4e10, block_len=2^28, M(y) int32, "
                          "64-bit quotient path, sieve+scan+update+resolve"),
    "1e12": dict(n=[10**12], u=10**8, block_len=1 << 24, pin=None,
                 workload="single query n=1e12, u=1e8, block_len=2^24"),
}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--mode", choices=["auto", "replicas", "shard"], default="auto",
                    help="N > 1: shard one target over the ranks by y-windows (auto, strong "
                         "scaling) or run independent replicas (weak scaling)")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="1e16")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the timed oracle sample (cpu_baseline key)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the M(10^18) wall time and the serving measurement")
    ap.add_argument("--serve-sample", type=int, default=2000,
                    help="queries of the seeded 10^4-query serving stream measured (extra key; "
                         "the one-plan-per-query baseline of all 10^4 alone would take about "
                         "5.5 minutes)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; independent replicas)
# ---------------------------------------------------------------------------
def dist_init(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle sample (the reference arm and the cpu_baseline key)
# ---------------------------------------------------------------------------
def oracle_sample(cfg, budget_s: float = 15.0):
    """Times the plain oracle computing array entries M(floor(n/x)) of the
    workload, smallest k first (x = X, X-1, ...), until `budget_s` elapses.
    Returns (terms/s, seconds, entries, terms) where terms are the method's
    closed-form update terms of those entries."""
    import oracle
    import paper_1108_0135_gb300 as pm

    oracle.build()
    n, u = cfg["n"][0], cfg["u"]
    X = n // u
    t0 = time.perf_counter()
    terms = 0
    done = 0
    x = X
    while x >= 1 and time.perf_counter() - t0 < budget_s:
        k = n // x
        oracle.mertens(k, L=max(math.isqrt(k) + 1, 10**6))
        s = math.isqrt(k)
        jlo, jhi = k // u + 1, k // (s + 1)
        terms += s + max(0, jhi - jlo + 1)
        done += 1
        x -= 1
    dt = time.perf_counter() - t0
    _ = pm  # the closed form above is the one mertens_describe reports
    return terms / dt, dt, done, terms


def oracle_sample_all_cores(cfg, budget_s: float = 15.0, workers: int = 0):
    """The same sample on every host core: threads take entries x = X, X-1, ...
    from a shared cursor and call the oracle (a C call through ctypes, which
    releases the interpreter lock), until `budget_s` elapses.  Returns
    (terms/s, seconds, entries, terms, threads)."""
    import oracle

    oracle.build()
    workers = workers or os.cpu_count() or 1
    n, u = cfg["n"][0], cfg["u"]
    X = n // u
    lock = threading.Lock()
    state = {"x": X, "terms": 0, "done": 0}
    t0 = time.perf_counter()

    def work():
        while time.perf_counter() - t0 < budget_s:
            with lock:
                x = state["x"]
                if x < 1:
                    return
                state["x"] = x - 1
            k = n // x
            oracle.mertens(k, L=max(math.isqrt(k) + 1, 10**6))
            s = math.isqrt(k)
            jlo, jhi = k // u + 1, k // (s + 1)
            with lock:
                state["terms"] += s + max(0, jhi - jlo + 1)
                state["done"] += 1

    threads = [threading.Thread(target=work) for _ in range(workers)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    dt = time.perf_counter() - t0
    return state["terms"] / dt, dt, state["done"], state["terms"], workers


def run_reference(args, world, rank):
    cfg = CONFIGS[args.config]
    if rank != 0:
        return
    samples = []
    for _ in range(args.warmup):
        oracle_sample_all_cores(cfg, budget_s=2.0)
    total_terms, total_s, entries, nth = 0, 0.0, 0, 1
    for _ in range(args.steps):
        _, dt, done, terms, nth = oracle_sample_all_cores(cfg, budget_s=10.0)
        total_terms += terms
        total_s += dt
        entries += done
        samples.append(dt)
    value = total_terms / total_s
    n, u = cfg["n"][0], cfg["u"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "update terms/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": cfg["workload"], "n": n, "u": u,
                   "block_len": cfg["block_len"], "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": "update terms/s", "cores": nth, "kind": "oracle",
                         "sample": f"{entries} array entries M(floor(n/x)), x = X, X-1, ... of "
                                   f"n={n}, u={u}, each by the oracle's Sec. 2 recursion, one "
                                   f"entry per call on {nth} threads (~10 s per step); terms = "
                                   f"the method's closed-form update terms of those entries"},
        "e2e": {"value": value, "unit": "update terms/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def serving_measure(sample: int):
    """Batched-query latency: the first `sample` queries of the seeded
    10^4-query stream (n log-uniform in [10^10, 10^16]) through the native
    continuous-batching server, closed loop (all submitted at once) and open
    loop (Poisson arrivals at 0.8 x the closed-loop rate), against the same
    queries run one plan each; every answer of every mode equals the
    one-plan-per-query answer."""
    import paper_1108_0135_gb300 as pm
    from paper_1108_0135_gb300 import serve, workloads

    _, ns = workloads.serving_stream(seed=20261203, count=10_000)
    ns = [int(v) for v in ns[:sample]]
    one = serve.run_one_per_plan(ns)
    closed = serve.run_stream(ns)
    assert closed["answers"] == one["answers"]
    rate = 0.8 * closed["queries_per_s"]
    arr = np.cumsum(np.random.default_rng(20261203).exponential(1.0 / rate, size=len(ns)))
    opened = serve.run_stream(ns, arrivals_s=arr)
    assert opened["answers"] == one["answers"]
    # the same stream with a resident M(y) table (y <= 2^34, sieved once and
    # timed separately): batches run update + resolve only
    import torch
    t0 = time.perf_counter()
    table = pm.mertens_table_create(1 << 34, 10**16)
    torch.cuda.synchronize()
    t_table = time.perf_counter() - t0
    tinfo = pm.mertens_table_info(table)
    try:
        tab = serve.run_stream(ns, table=table)
        assert tab["answers"] == one["answers"]
        rate_t = 0.8 * tab["queries_per_s"]
        arr_t = np.cumsum(np.random.default_rng(20261203).exponential(1.0 / rate_t,
                                                                       size=len(ns)))
        tab_open = serve.run_stream(ns, arrivals_s=arr_t, table=table)
        assert tab_open["answers"] == one["answers"]
    finally:
        pm.mertens_table_destroy(table)
    return {
        "sample": f"first {len(ns)} of the seeded 10^4-query stream, n log-uniform in "
                  f"[1e10, 1e16] (every answer checked against one plan per query)",
        "one_plan_per_query_qps": one["queries_per_s"],
        "closed_loop": {"qps": closed["queries_per_s"], "p50_s": closed["p50_s"],
                        "p99_s": closed["p99_s"], "batches": closed["stats"]["batches"],
                        "max_batch": closed["stats"]["max_batch_seen"],
                        "max_inflight": closed["stats"]["max_inflight"]},
        "open_loop": {"rate_qps": rate, "qps": opened["queries_per_s"],
                      "p50_s": opened["p50_s"], "p99_s": opened["p99_s"]},
        "batched_over_one_per_plan": closed["queries_per_s"] / one["queries_per_s"],
        "resident_table": {
            "y_max": tinfo["y_max"], "n_max": tinfo["n_max"], "device_bytes": tinfo["bytes"],
            "build_s": t_table,
            "closed_loop": {"qps": tab["queries_per_s"], "p50_s": tab["p50_s"],
                            "p99_s": tab["p99_s"], "batches": tab["stats"]["batches"]},
            "open_loop": {"rate_qps": rate_t, "qps": tab_open["queries_per_s"],
                          "p50_s": tab_open["p50_s"], "p99_s": tab_open["p99_s"]},
            "over_one_per_plan": tab["queries_per_s"] / one["queries_per_s"],
        },
    }


def run_sharded(args, world, rank, local):
    """One target over `world` ranks: each rank runs its y-window (window
    plan), the windows' carries and sums are exchanged (all-gather of mu sums,
    all-reduce of the entries' sums), rank 0 resolves.  Strong scaling."""
    import torch

    import paper_1108_0135_gb300 as pm
    from paper_1108_0135_gb300 import shard

    cfg = CONFIGS[args.config]
    pm.load()
    pm.use_torch_allocator()
    stream = torch.cuda.current_stream()
    n, u, L = cfg["n"][0], cfg["u"], cfg["block_len"]
    info = pm.mertens_describe(n, u)
    terms = info["direct_terms"] + info["gathered_terms"]
    device = torch.device("cuda", local) if world > 1 else None
    tgt = shard.ShardedTarget(n, u, L, rank, world, device)
    for _ in range(max(args.warmup, 1)):
        arr = tgt.step(stream)
    if rank == 0 and cfg["pin"] is not None and int(arr[0]) != cfg["pin"]:
        raise SystemExit(f"wrong result: M({n}) = {int(arr[0])}, expected {cfg['pin']}")
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        arr = tgt.step(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    clk = clocks.stop()
    # each step ends with the resolved array read to the host, so the device
    # interval between the events spans the whole step
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = max_over_ranks(ms, world)
    wall_max = max_over_ranks(wall_ms, world)
    if rank == 0 and cfg["pin"] is not None:
        assert int(arr[0]) == cfg["pin"]
    # this rank's window, kernel by kernel with the library's phase events
    phases = {}
    if tgt.plan:
        pm.mertens_plan_set_profiling(tgt.plan, True)
        pm.mertens_run(tgt.plan, stream)
        torch.cuda.synchronize()
        st = pm.mertens_run_stats_get(tgt.plan)
        phases = {"mu_sieve": st["sieve_ms"], "seg_carry": st["scan_ms"],
                  "update_dense": st["dense_ms"], "update_gathered": st["gather_ms"]}
        kernels = int(st["kernels"])
        peaks, _ = load_peaks()
        roofs = rooflines(phases, st, peaks, int(st["blocks"]), pm.mertens_probe_int_peaks(stream))
    else:
        kernels, roofs = 0, {}
    window = tgt.window
    tgt.close()
    X = info["X"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": terms / (ms_max / 1e3), "unit": "update terms/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": cfg["workload"], "n": n, "u": u, "block_len": L,
                       "X": info["X"], "terms_per_step": terms,
                       "l2": "inputs larger than L2 (M blocks of 512 MiB)",
                       "parallelism": f"y-windows over {world} ranks: window plans, all-gather "
                                      f"of mu sums, all-reduce of entry sums, resolve on rank 0"},
            "wall_time_s": ms_max / 1e3,
            "host_wall_ms_per_step": wall_max,
            "rank0_window": list(window),
            "rank0_phases_ms": {k: round(v, 3) for k, v in phases.items()},
            "clocks": clk,
            # every step reads the window's mu sum (8 bytes) and, on rank 0,
            # the resolved array to the host; the exchange stays on the device:
            # the host wall time is the end-to-end figure
            "e2e": {"value": terms / (wall_max / 1e3), "unit": "update terms/s",
                    "h2d_bytes_per_step": 8 * world, "d2h_bytes_per_step": 8 * X + 8,
                    "ms_per_step": wall_max},
            "gpu_launches": (kernels + 1) * args.steps,
            "roofline": (roofs[max(roofs, key=lambda k: phases[k])] if roofs else None),
            "rooflines_rank0": roofs,
            "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)


def run_native(args, world, rank, local):
    import torch

    import paper_1108_0135_gb300 as pm

    cfg = CONFIGS[args.config]
    pm.load()
    pm.use_torch_allocator()
    stream = torch.cuda.current_stream()
    n_list, u, L = cfg["n"], cfg["u"], cfg["block_len"]

    plan = pm.mertens_plan(n_list, u, L)
    info = pm.mertens_plan_info(plan, 0)
    terms = info["direct_terms"] + info["gathered_terms"]
    # warm-up (first run also builds the n-independent divisor table)
    for _ in range(max(args.warmup, 1)):
        pm.mertens_run(plan, stream)
    m_n, _ = pm.mertens_result(plan, 0)
    if cfg["pin"] is not None and m_n != cfg["pin"]:
        raise SystemExit(f"wrong result: M({n_list[0]}) = {m_n}, expected {cfg['pin']}")

    # timed region: K steps (whole runs replayed from the plan's CUDA graph),
    # CUDA events on the launching stream, clocks sampled meanwhile
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        pm.mertens_run(plan, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    m_chk, _ = pm.mertens_result(plan, 0)
    assert m_chk == m_n
    # the same K steps launched kernel by kernel with the library's phase
    # events on the same stream: per-kernel-class times for the rooflines
    pm.mertens_plan_set_profiling(plan, True)
    torch.cuda.synchronize()
    pe0 = torch.cuda.Event(enable_timing=True)
    pe1 = torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(args.steps):
        pm.mertens_run(plan, stream)
    pe1.record(stream)
    torch.cuda.synchronize()
    ms_eager = pe0.elapsed_time(pe1) / args.steps
    stats = pm.mertens_run_stats_get(plan)
    m_chk, _ = pm.mertens_result(plan, 0)
    assert m_chk == m_n
    pm.mertens_destroy(plan)
    ms_max = max_over_ranks(ms, world)
    value = terms * world / (ms_max / 1e3)

    # M(10^18) wall time (the metric's second figure), one warm run timed
    extra = {}
    if world == 1 and args.config == "1e16" and not args.no_extra:
        p18 = pm.mertens_plan([10**18])
        i18 = pm.mertens_plan_info(p18, 0)
        pm.mertens_run(p18, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pm.mertens_run(p18, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        m18, _ = pm.mertens_result(p18, 0)
        pm.mertens_destroy(p18)
        t18 = e0.elapsed_time(e1) / 1e3
        extra["M_1e18"] = {"M": m18, "expected_table1": -46758740, "wall_time_s": t18,
                           "u": i18["u"], "X": i18["X"],
                           "update_terms_per_s": (i18["direct_terms"] + i18["gathered_terms"])
                           / t18}
        extra["batch_64_close_1e17"] = batch_measure(stream)
        extra["u128_window_1e20"] = window_measure(stream)
        extra["serving"] = serving_measure(args.serve_sample)


    # e2e: the user call with host inputs and host results, every step
    host_out = torch.empty(info["X"], dtype=torch.int64, pin_memory=True)
    out_np = host_out.numpy()
    e2e_ms = []
    h2d = d2h = 0
    for it in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p2 = pm.mertens_plan(n_list, u, L)
        pm.mertens_run(p2, stream)
        m2 = pm.mertens_result_into(p2, 0, out_np)
        st2 = pm.mertens_run_stats_get(p2)
        pm.mertens_destroy(p2)
        dt = time.perf_counter() - t0
        assert m2 == m_n
        if it > 0:  # first iteration warms the allocator cache
            e2e_ms.append(dt * 1e3)
        h2d, d2h = st2["h2d_bytes"] + 16 * len(n_list), st2["d2h_bytes"]
    e2e_ms_max = max_over_ranks(float(np.mean(e2e_ms)), world) if e2e_ms else float("nan")
    e2e_value = terms * world / (e2e_ms_max / 1e3) if e2e_ms else None

    # roofline of the dominant kernel class
    peaks, peak_src = load_peaks()
    phases = {"mu_sieve": stats["sieve_ms"], "seg_carry": stats["scan_ms"],
              "update_dense": stats["dense_ms"], "update_gathered": stats["gather_ms"],
              "resolve": stats["resolve_ms"]}
    ipk = pm.mertens_probe_int_peaks(stream)
    roofs = rooflines(phases, stats, peaks, int(stats["blocks"]), ipk)
    dom = max(roofs, key=lambda k: phases[k])
    roof = roofs[dom]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, done, tms = oracle_sample(cfg, budget_s=15.0)
        cpu = {"value": v, "unit": "update terms/s", "cores": 1, "kind": "oracle",
               "sample": f"{done} array entries M(floor(n/x)), x = X, X-1, ... of the same "
                         f"workload by the oracle's Sec. 2 recursion ({dt:.1f} s); terms = "
                         f"the method's closed-form update terms of those entries"}
        try:
            va, dta, donea, _, nth = oracle_sample_all_cores(cfg, budget_s=15.0)
            cpu["all_cores"] = {
                "value": va, "cores": nth,
                "sample": f"{donea} entries of the same sequence, one oracle call per entry on "
                          f"{nth} threads ({dta:.1f} s)"}
        except Exception as exc:  # the single-core figure stands on its own
            cpu["all_cores"] = {"error": str(exc)[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "update terms/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": cfg["workload"], "n": n_list[0], "u": u,
                       "block_len": L, "X": info["X"], "terms_per_step": terms,
                       "M_n": m_n, "l2": "inputs larger than L2 (M block 1 GiB, "
                                         "divisor table 1.3 GB per step)",
                       "parallelism": f"{world} independent replicas"},
            "wall_time_s": ms_max / 1e3,
            # `value` counts the paper's direct + gathered terms (closed form per
            # entry); the kernels reach the same sums through the mu-form, which
            # executes one quotient per squarefree y below the dense cut-off and
            # one per gathered j above it, less the gathered terms entry 2x takes
            # from entry x's even j (floor(floor(n/x)/2j) = floor(floor(n/2x)/j)):
            "terms_executed_per_step": dense_evaluated(stats) + stats["gather_j_exec"],
            "gathered_terms_shared_per_step": stats["gather_j"] - stats["gather_j_exec"],
            "phases_ms": {k: round(v, 3) for k, v in phases.items()},
            "y_sieved_per_s": stats["y_sieved"] * world / (ms_max / 1e3),
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "update terms/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms_max},
            "gpu_launches": int(stats["kernels"]) * args.steps,
            "roofline": roof,
            "rooflines": roofs,
            "phase_timing": f"library CUDA events on the launching stream, {args.steps} steps "
                            f"launched kernel by kernel right after the timed graph-replay "
                            f"steps ({ms_eager:.2f} ms/step that way)",
            "extra": extra,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def _timed_run(plan, stream, repeats: int = 1):
    """Seconds of warm mertens_run calls (CUDA events on the launching
    stream): one untimed run, then `repeats` timed ones; returns the list."""
    import torch
    import paper_1108_0135_gb300 as pm
    pm.mertens_run(plan, stream)
    torch.cuda.synchronize()
    out = []
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pm.mertens_run(plan, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1) / 1e3)
    return out


def batch_measure(stream, repeats: int = 3):
    """64 close targets 10^17 + i 10^9 in one plan (one sieve pass): wall time
    (median of `repeats` warm runs) and update terms/s; M(10^17) from Table 1
    checked; targets 0, 1 and 63 alone, with the batch's u, give the same
    whole arrays; one target alone with its own u timed beside it."""
    import paper_1108_0135_gb300 as pm
    from paper_1108_0135_gb300 import workloads
    cfg = workloads.BATCH_1E17
    ns = cfg["n"]
    plan = pm.mertens_plan(ns, cfg["u"], 0)
    infos = [pm.mertens_plan_info(plan, i) for i in range(len(ns))]
    ts = _timed_run(plan, stream, repeats)
    m0, _ = pm.mertens_result(plan, 0)
    batched = {i: pm.mertens_result(plan, i, entries=True) for i in (0, 1, 63)}
    pm.mertens_destroy(plan)
    assert m0 == -21830254, m0
    for i, (mi, arr) in batched.items():
        pa = pm.mertens_plan([ns[i]], infos[i]["u"], 0)
        pm.mertens_run(pa, stream)
        ma, arra = pm.mertens_result(pa, 0, entries=True)
        pm.mertens_destroy(pa)
        assert ma == mi and np.array_equal(arra, arr), i
    t = float(np.median(ts))
    terms = sum(i["direct_terms"] + i["gathered_terms"] for i in infos)
    p1 = pm.mertens_plan([ns[0]])
    t1s = _timed_run(p1, stream, repeats)
    pm.mertens_destroy(p1)
    t1 = float(np.median(t1s))
    return {"targets": len(ns), "wall_time_s": t, "wall_time_runs_s": ts,
            "update_terms_per_s": terms / t,
            "queries_per_s": len(ns) / t, "u": infos[0]["u"], "X_each": infos[0]["X"],
            "M_n0": m0, "expected_table1": -21830254,
            "alone_equals_batched": [0, 1, 63],
            "one_target_alone_s": t1, "one_target_alone_runs_s": t1s,
            "alone_x64_over_batch": 64 * t1 / t,
            "alone_x64_over_batch_range": [64 * min(t1s) / max(ts), 64 * max(t1s) / min(ts)]}


def window_measure(stream):
    """Two-word target n = 10^20 (u ~ n^(2/3)): the update of 64 sieve blocks of
    2^28 y from y = 10^13 (window plan: carry left symbolic), y sieved/s and
    entries scanned/s."""
    import paper_1108_0135_gb300 as pm
    from paper_1108_0135_gb300 import workloads
    cfg = workloads.WINDOW_1E20
    plan = pm.mertens_plan_window(cfg["n"], cfg["y_first"], cfg["y_last"], cfg["u"],
                                  cfg["block_len"])
    info = pm.mertens_plan_info(plan, 0)
    t = _timed_run(plan, stream)[0]
    S, coef, mu = pm.mertens_window_result(plan, 0)
    pm.mertens_destroy(plan)
    ny = cfg["y_last"] - cfg["y_first"] + 1
    terms = int(np.count_nonzero(coef))
    gathered = int(coef.astype(np.uint64).sum(dtype=np.uint64))
    return {"n": str(cfg["n"][0]), "u": cfg["u"], "X": info["X"], "y_first": cfg["y_first"],
            "blocks": 64, "y": ny, "wall_time_s": t, "y_sieved_per_s": ny / t,
            "entries_scanned_per_s": info["X"] * 64 / t, "gathered_terms": gathered,
            "entries_with_terms": terms, "mu_sum": mu}


# From ncu captures of the current kernel versions on the n = 10^16 workload
# (one GB300, --clock-control none), per kernel class:
#   dram_bytes_per_step: dram__bytes_read.sum + dram__bytes_write.sum summed
#     over all of the class's launches in one run (a run of the capture, or
#     one captured launch times the launches per run where every launch does
#     the same work per y), None when a kernel of the class changed since;
#   issue_active: smsp__issue_active.avg.pct_of_peak_sustained_active of the
#     class's main kernel (share of cycles a scheduler issued an instruction);
#   pipe: the busiest pipe of that kernel and its share of active cycles.
NCU = {
    "mu_sieve": {"kernel": "mu_sieve_t2_kernel", "dram_bytes_per_step": 72.3e9,
                 "issue_active": 0.666, "pipe": ("alu", 0.436)},
    "update_dense": {"kernel": "dense_update_kernel", "dram_bytes_per_step": 0.87e9,
                     "issue_active": 0.446, "pipe": ("fmaheavy", 0.799)},
    "update_gathered": {"kernel": "gather_tile_kernel", "dram_bytes_per_step": 13.9e9,
                        "issue_active": 0.830, "pipe": ("fmaheavy", 0.668)},
}
# Issue slots of the chip: 152 SMs x 4 schedulers x one warp instruction per
# clock at the maximum SM clock.
ISSUE_PEAK_WARP_INSTR_PER_S = 152 * 4 * 2070e6

SIX_OVER_PI2 = 6.0 / math.pi ** 2


def dense_evaluated(stats):
    """Squarefree y the dense kernel evaluates: (6/pi^2) of the summed dense
    y-ranges, less the odd squarefree y (8/pi^2 of the odd y) that entries 2x
    take from entries x (mu(y) floor(floor(n/2x)/y) = -mu(2y) floor(floor(n/x)/2y))."""
    return SIX_OVER_PI2 * stats["dense_y"] - (4.0 / 3.0) * SIX_OVER_PI2 * stats["dense_odd_skip"]


def rooflines(phases, stats, peaks, nblocks, ipk):
    """Roofline records per kernel class of the timed region.

    Every class here is bound by integer issue (no tensor cores, no floating
    point contraction; HBM traffic is about 2 B per sieved y).  MEASURED_PEAKS
    holds no integer figure, so `peak` is the speed of the class's own inner
    step, measured on this device by mertens_probe_int_peaks (ipk: independent
    chains of that step on every SM) -- `frac` is the fraction of that
    inner-step speed, not of a chip pipe peak.  Beside it, `issue` gives the
    ncu issue-active share of the class's main kernel and its busiest pipe
    (NCU above), against the chip's issue slots.
      update_dense: the update's inner step acc += mulhi64(m, 2k) >> l, in
        terms/s.  Units: squarefree y the kernel evaluates (dense_evaluated).
      update_gathered: one term per gathered j evaluated (entry 2x takes
        part of its terms from entry x's even j, so fewer than the method's
        gathered terms), against the faster of that step and the
        shared-memory gather's float-estimate quotient step (the tile kernel
        takes the latter, the global path the former).
      mu_sieve: 32-bit ALU lane operations/s (LOP3 + IADD3 chains).
        Algorithmic operations: one per sieve update (y, p | y or p^2 | y
        for every sieving prime p) plus two per y (decision + scan add).
    `achieved` and `traffic` are per step (all launches of the class)."""
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    mulhi_peak = ipk["mulhi_terms_per_s"] / 1e12
    alu_peak = 2.0 * ipk["alu_pairs_per_s"] / 1e12
    gather_peak = max(ipk["mulhi_terms_per_s"], ipk.get("fquot_terms_per_s", 0.0)) / 1e12
    work = {
        "mu_sieve": (stats["sieve_updates"] + 2.0 * stats["y_sieved"], alu_peak, "T int-op/s",
                     "inner-step probe: LOP3+IADD3 chains on all SMs, 2 ops per pair"),
        "update_dense": (dense_evaluated(stats), mulhi_peak, "T mulhi-terms/s",
                         "inner-step probe: acc += mulhi64(m,2k) >> l chains on all SMs"),
        "update_gathered": (float(stats["gather_j_exec"]), gather_peak, "T terms/s",
                            "inner-step probe: the faster of the mulhi64 step and the "
                            "float-estimate quotient step, chains on all SMs"),
    }
    out = {}
    for k, (v, peak, unit, src) in work.items():
        ms = phases.get(k, 0.0)
        if ms <= 0:
            continue
        achieved = v / (ms / 1e3) / 1e12
        nc = NCU[k]
        out[k] = {"bound": "alu", "kernel": k, "achieved": achieved, "peak": peak,
                  "unit": unit, "frac": achieved / peak,
                  "frac_of": "the class's inner-step speed measured by the probe",
                  "traffic": nc["dram_bytes_per_step"], "traffic_per": "step",
                  "issue": {"kernel": nc["kernel"], "ncu_issue_active": nc["issue_active"],
                            "busiest_pipe": nc["pipe"][0], "pipe_active": nc["pipe"][1],
                            "peak_warp_instr_per_s": ISSUE_PEAK_WARP_INSTR_PER_S},
                  "peak_source": f"{src} ({ipk['sms']} SMs, max SM clock {sm_mhz:.0f} MHz)"}
    return out


def main():
    args = parse_args()
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, world, rank)
        return
    world, rank, local = dist_init(args)
    try:
        shard = args.mode == "shard" or (args.mode == "auto" and world > 1)
        if shard:
            run_sharded(args, world, rank, local)
        else:
            run_native(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
