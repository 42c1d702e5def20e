"""Served workload: a seeded Poisson stream of generation requests replayed
in real time against one gc_server (continuous batching), reporting p50/p99
latency and jobs/s.

    python -m paper_1507_05398_gb300.serve [--requests 10000] [--load 0.8]

The arrival rate is `load` times the server's measured capacity (a burst of
the same request mix submitted at once).  Latency = completion seen by the
host - arrival time (it includes waiting for admission).
"""
from __future__ import annotations

import argparse
import json
import statistics
import time

from .gc import Server
from .workloads import batch_instances, serve_requests


def _drain(srv, inflight, done_times, fetch=False):
    for rid in srv.poll():
        done_times[inflight.pop(rid)] = time.perf_counter()
        if fetch:
            srv.fetch(rid)
        srv.release(rid)


def capacity(srv, probs) -> float:
    """Jobs/s when the whole burst is available at once."""
    inflight, done, pending = {}, {}, list(enumerate(probs))
    t0 = time.perf_counter()
    while pending or inflight:
        while pending:
            k, p = pending[0]
            rid = srv.submit(*p)
            if rid is None:
                break
            inflight[rid] = k
            pending.pop(0)
        _drain(srv, inflight, done)
        time.sleep(0.0001)
    return len(probs) / (time.perf_counter() - t0)


def replay(srv, stream):
    """stream: [(arrival_s, problem)]; returns per-request latencies (s)."""
    inflight, done, pending = {}, {}, []
    arrivals = [t for t, _ in stream]
    nxt = 0
    t0 = time.perf_counter()
    while nxt < len(stream) or pending or inflight:
        now = time.perf_counter() - t0
        while nxt < len(stream) and stream[nxt][0] <= now:
            pending.append(nxt)
            nxt += 1
        while pending:
            k = pending[0]
            rid = srv.submit(*stream[k][1])
            if rid is None:
                break
            inflight[rid] = k
            pending.pop(0)
        _drain(srv, inflight, done)
        time.sleep(0.0001)
    makespan = max(done.values()) - t0
    lat = [done[k] - (t0 + arrivals[k]) for k in range(len(stream))]
    return lat, makespan


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--seed", type=int, default=1507)
    ap.add_argument("--groups", type=int, default=0)
    args = ap.parse_args()
    with Server(max_n=28, ngroups=args.groups, pool_bytes=8 << 30, queue_capacity=2048) as srv:
        # capacity on the same mix (95% batch distribution, 5% large)
        probe = [p for _, p in serve_requests(1024, args.seed + 1, 1.0)]
        cap = capacity(srv, probe)
        rate = args.load * cap
        stream = serve_requests(args.requests, args.seed, rate)
        lat, makespan = replay(srv, stream)
    lat_ms = sorted(1e3 * x for x in lat)
    q = lambda f: lat_ms[min(len(lat_ms) - 1, int(f * len(lat_ms)))]
    print(json.dumps({
        "workload": f"served: {args.requests} seeded Poisson requests (seed {args.seed}), 95% "
                    "n~U{14..24} d~U{3..8} any order (25% constant weight), 5% n~U{26..28} "
                    "d~U{3,4}",
        "capacity_jobs_per_s": cap, "load": args.load, "rate_jobs_per_s": rate,
        "jobs_per_s": args.requests / makespan, "makespan_s": makespan,
        "latency_ms": {"p50": q(0.50), "p90": q(0.90), "p99": q(0.99), "max": lat_ms[-1],
                       "mean": statistics.mean(lat_ms)},
    }))


if __name__ == "__main__":
    main()
