"""Request streams through the native continuous-batching server.

The server itself (admission, batching, streams, memory budget) is native
code in libmertens (``mertens_server_*``); this module only submits a stream
of queries -- all at once (closed loop) or at given arrival times (open loop)
-- collects the answers and the server's own submit/answer timestamps, and
times the one-query-per-plan alternative for comparison.
"""
from __future__ import annotations

import time

import numpy as np

from . import _lib as L


def run_stream(ns, arrivals_s=None, device=0, max_inflight=0, max_batch=0, mem_budget=0,
               table=0):
    """Submits every n (at arrivals_s[i] seconds after the start if given,
    else all at once), waits for all answers.  Returns a dict with the
    answers, per-query latencies (s), throughput and the server's stats.
    With a resident table handle, batches that fit it are planned on it."""
    srv = L.mertens_server_create(device, mem_budget, max_inflight, max_batch)
    try:
        if table:
            L.mertens_server_use_table(srv, table)
        tickets = []
        t0 = time.perf_counter()
        if arrivals_s is None:
            for n in ns:
                tickets.append(L.mertens_server_submit(srv, int(n)))
        else:
            order = np.argsort(arrivals_s, kind="stable")
            for i in order:
                delay = float(arrivals_s[i]) - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                tickets.append((int(i), L.mertens_server_submit(srv, int(ns[i]))))
            tickets = [t for _, t in sorted(tickets)]
        answers = [L.mertens_server_wait(srv, t) for t in tickets]
        t_end = time.perf_counter()
        times = [L.mertens_server_times(srv, t) for t in tickets]
        stats = L.mertens_server_stats_get(srv)
    finally:
        L.mertens_server_destroy(srv)
    lat = np.array([(d - s) / 1e9 for s, d in times])
    first = min(s for s, _ in times)
    last = max(d for _, d in times)
    return {
        "answers": answers,
        "latency_s": lat,
        "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)),
        "makespan_s": (last - first) / 1e9,
        "wall_s": t_end - t0,
        "queries_per_s": len(ns) / ((last - first) / 1e9),
        "stats": stats,
    }


def run_one_per_plan(ns, stream=None):
    """The same queries one at a time, each its own plan and run."""
    t0 = time.perf_counter()
    out = []
    for n in ns:
        out.append(L.mertens(int(n), stream=stream))
    dt = time.perf_counter() - t0
    return {"answers": out, "wall_s": dt, "queries_per_s": len(ns) / dt}
