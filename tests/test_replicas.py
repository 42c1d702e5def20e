"""Replicas across ranks (world_size 2, gloo on CPU): the batch is split by
estimated work with no job lost or duplicated, every rank's share is
computed (here by the oracle, standing in for one GPU each), results and the
max-over-ranks timing are gathered."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1507_05398_gb300.replicas import job_cost, shard
from paper_1507_05398_gb300.workloads import batch_instances


def test_shard_covers_every_job_once_and_balances():
    probs = batch_instances(512, 1507)
    for world in (1, 2, 3, 8):
        parts = shard(probs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(probs)))
        loads = [sum(job_cost(*probs[i]) for i in p) for p in parts]
        assert max(loads) <= 1.5 * (sum(loads) / world) + max(job_cost(*p) for p in probs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, probs, q):
    import torch.distributed as dist

    import oracle
    from paper_1507_05398_gb300.replicas import gather_results, max_over_ranks, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard(probs, world)[rank]
    local = {i: oracle.greedy_ball(*probs[i]).tolist() for i in mine}
    merged = gather_results(local, world, rank)
    slowest = max_over_ranks(float(rank + 1), world)
    if rank == 0:
        q.put((merged, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_replicas():
    probs = [p for p in batch_instances(64, 7) if p[0] <= 16][:12]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, probs, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, slowest = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    assert slowest == 2.0
    assert sorted(merged) == list(range(len(probs)))
    for i, p in enumerate(probs):
        assert merged[i] == oracle.greedy_ball(*p).tolist()
