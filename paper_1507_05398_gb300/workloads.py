"""Seeded synthetic workloads (the problem instances only; no arithmetic of
the method lives here).  Shared by the tests, the benchmark and the request
server, so every side draws exactly the same instances.

Every instance is fully determined by (n, d, ordering, weight): there is no
dataset.  Draws use numpy's PCG64 generator.
"""
from __future__ import annotations

import numpy as np

ORDER_NAMES = ("lex", "gray", "grlex", "grevlex")


def batch_instances(count: int = 512, seed: int = 1507):
    """Batched workload: n ~ U{14..24}, d ~ U{3..8}, ordering ~ U{4}; with
    probability 0.25 constant weight w ~ U{3..floor(n/2)}, else no weight.
    Returns a list of (n, d, ordering, weight)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        n = int(rng.integers(14, 25))
        d = int(rng.integers(3, 9))
        o = ORDER_NAMES[int(rng.integers(0, 4))]
        w = int(rng.integers(3, n // 2 + 1)) if rng.random() < 0.25 else -1
        out.append((n, d, o, w))
    return out


def serve_requests(count: int = 10000, seed: int = 1507, rate_per_s: float = 1000.0):
    """Served workload: Poisson arrivals at rate_per_s; 95% of requests drawn
    like batch_instances, 5% with n ~ U{26..28}, d ~ U{3..4}, no weight.
    Returns a list of (arrival_time_s, (n, d, ordering, weight))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        if rng.random() < 0.05:
            n = int(rng.integers(26, 29))
            d = int(rng.integers(3, 5))
            o = ORDER_NAMES[int(rng.integers(0, 4))]
            w = -1
        else:
            n = int(rng.integers(14, 25))
            d = int(rng.integers(3, 9))
            o = ORDER_NAMES[int(rng.integers(0, 4))]
            w = int(rng.integers(3, n // 2 + 1)) if rng.random() < 0.25 else -1
        out.append((t, (n, d, o, w)))
    return out
