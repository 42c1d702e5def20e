"""Measured autotuning (gc_autotune) and the tuning cache."""
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
