"""Measured autotuning (gc_autotune, gc_batch_autotune) and the tuning cache."""
import hashlib
import json
import os
import statistics

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_autotune_records_and_is_used(tmp_path):
    import paper_1507_05398_gb300 as G
    cache = tmp_path / "tune.txt"
    G.set_tune_cache(str(cache))
    try:
        best, ms = G.autotune(17, 4, "gray")
        assert best.strategy in (1, 2) and ms > 0
        lines = cache.read_text().strip().splitlines()
        assert len(lines) == 1 and lines[0].split()[:5] == ["17", "4", "1", "-1", "0"]
        p = G.plan(17, 4, "gray")
        assert (p.strategy, p.survivor_target, p.grid) == (best.strategy, best.survivor_target,
                                                           best.grid)
        code = G.generate(17, 4, "gray").cpu().numpy().view(np.uint32)
        assert code.tolist() == oracle.greedy_ball(17, 4, "gray").tolist()
        # a self-orthogonal problem is never tuned onto the bitmap strategy
        best2, _ = G.autotune(16, 4, "lex", constraint="self_orthogonal")
        assert best2.strategy == 1
    finally:
        G.set_tune_cache(None)
    assert G.plan(17, 4, "gray").grid > 0


def _batch_ms(G, probs, reps=3):
    import torch
    b = G.BatchBuffers(probs)
    b.launch()
    torch.cuda.synchronize()
    g = b.capture()
    ts = []
    for _ in range(reps + 1):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        e.record()
        e.synchronize()
        ts.append(a.elapsed_time(e))
    return statistics.median(ts[1:]), b.results()


def test_batch_autotune_512_instances(tmp_path):
    """The 512 seeded batch instances with their costliest distinct problems
    tuned where they run (a group of the batch's CTAs): every code still
    equals the oracle's stored digest, and the tuned batch is not slower than
    the cost-model plan (within timing noise)."""
    import paper_1507_05398_gb300 as G
    from paper_1507_05398_gb300.workloads import batch_instances
    probs = batch_instances(512, 1507)
    rows = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "batch_expected.json")))["codes"]
    base_ms, _ = _batch_ms(G, probs)
    cache = tmp_path / "tune.txt"
    G.set_tune_cache(str(cache))
    try:
        tuned = G.batch_autotune(probs, max_jobs=12)
        assert tuned == 12
        entries = cache.read_text().strip().splitlines()
        assert len(entries) == 12 and all(e.split()[7] == "0" for e in entries)  # grid 0
        ms, res = _batch_ms(G, probs)
        print(f"512-instance batch: {base_ms:.2f} ms cost-model plan, {ms:.2f} ms tuned")
        for (n, d, o, w), row, (code, st) in zip(probs, rows, res):
            assert st.status == 0
            assert hashlib.sha256(code.astype("<u4").tobytes()).hexdigest() == row["sha256"]
        assert ms <= 1.10 * base_ms, (ms, base_ms)
    finally:
        G.set_tune_cache(None)
    with pytest.raises(G.GcError) as e:  # no cache installed
        G.batch_autotune(probs[:4])
    assert e.value.code == 1
