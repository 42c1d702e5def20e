"""Multi-GPU use: replicas only.  One code's sweep does not shard (every
acceptance must be visible before the frontier passes it), but independent
codes do: a batch or a request stream is split across ranks by estimated
work, each rank sweeps its share on its own GPU, and the results are
gathered.  No collective sits on the data path; torch.distributed is used
only to gather results and timings (gloo on CPU, nccl on GPUs).
"""
from __future__ import annotations

from math import comb


def job_cost(n: int, d: int, ordering: str = "lex", weight: int = -1) -> float:
    """Rough relative work of one code: the rank space plus the square of a
    code-size estimate (half the sphere-packing bound)."""
    N = (1 << n) if weight < 0 else comb(n, weight)
    t = max(0, (d - 1) // 2)
    bound = min(N, (1 << n) // sum(comb(n, k) for k in range(t + 1)))
    C = max(1.0, bound / 2.0)
    return float(N) + C * C / 64.0


def shard(problems, world: int):
    """Longest-first assignment of problems to `world` ranks: returns a list of
    index lists, one per rank, each in submission order."""
    order = sorted(range(len(problems)), key=lambda i: -job_cost(*problems[i]))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: load[k])
        parts[r].append(i)
        load[r] += job_cost(*problems[i])
    return [sorted(p) for p in parts]


def gather_results(local: dict, world: int, rank: int, group=None):
    """All ranks' {problem index: result} merged on every rank."""
    import torch.distributed as dist
    if world == 1:
        return dict(local)
    out = [None] * world
    dist.all_gather_object(out, local, group=group)
    merged = {}
    for part in out:
        merged.update(part)
    return merged


def max_over_ranks(value: float, world: int) -> float:
    """The slowest rank's time (the bench's timing rule)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
