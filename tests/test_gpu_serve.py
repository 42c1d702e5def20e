"""The request server (gc_server_*): requests submitted while others run are
admitted as pool space frees up, and each result equals the oracle's and the
result of the same request run alone."""
import time

import numpy as np
import pytest

import oracle
from paper_1507_05398_gb300.workloads import batch_instances

pytestmark = pytest.mark.gpu


def test_server_mix_equals_alone_and_oracle():
    import paper_1507_05398_gb300 as G
    probs = [p for p in batch_instances(512, 99) if p[0] <= 18][:60]
    probs += [(18, 3, "lex", -1), (16, 2, "gray", -1), (15, 1, "grlex", -1), (14, 9, "grevlex", 5)]
    alone = {}
    for p in probs[::7]:  # a sample run alone, before the server holds the SMs
        alone[p] = G.generate(*p).cpu().numpy().view(np.uint32)
    # a small pool and ring force admission to wait for releases
    results = {}
    with G.Server(max_n=20, ngroups=6, pool_bytes=8 << 20, queue_capacity=16) as srv:
        pending = list(enumerate(probs))
        inflight = {}
        t0 = time.time()
        while pending or inflight:
            assert time.time() - t0 < 120, "server made no progress"
            while pending:
                k, p = pending[0]
                rid = srv.submit(*p)
                if rid is None:
                    break
                inflight[rid] = (k, p)
                pending.pop(0)
            for rid in srv.poll():
                k, p = inflight.pop(rid)
                code, st = srv.fetch(rid)
                srv.release(rid)
                assert st.status == 0
                results[k] = code
            time.sleep(0.0002)
    for k, p in enumerate(probs):
        want = oracle.greedy_ball(*p)
        assert results[k].tolist() == want.tolist(), p
        if p in alone:
            assert alone[p].tolist() == results[k].tolist()


def test_server_restarts_after_idle_exit():
    import paper_1507_05398_gb300 as G
    with G.Server(max_n=16, ngroups=4, pool_bytes=1 << 20, queue_capacity=8,
                  idle_seconds=0.2) as srv:
        for round_ in range(2):
            rid = srv.submit(14, 3, "gray")
            t0 = time.time()
            while True:
                done = srv.poll()
                if rid in done:
                    break
                assert time.time() - t0 < 30
                time.sleep(0.001)
            code, st = srv.fetch(rid)
            srv.release(rid)
            assert code.tolist() == oracle.greedy_ball(14, 3, "gray").tolist()
            time.sleep(0.5)  # the device loop leaves; the next submit restarts it
