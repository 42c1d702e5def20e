"""Failure detection without a GPU fault: every device-side wait of the sweep
is bounded.  A host-side injection (GC_FAULT=wait) makes one group wait for a
CTA that does not exist; the wait must expire, the call must report
GC_ERR_TIMEOUT, and the same CUDA context must keep working afterwards."""
import os
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_context_survives():
    import paper_1507_05398_gb300 as G
    os.environ["GC_FAULT"] = "wait"
    try:
        t = time.time()
        with pytest.raises(G.GcError) as e:
            G.generate(15, 3, "lex")
        assert e.value.code == 5  # GC_ERR_TIMEOUT
        assert time.time() - t < 30
        # the grid sweep's barriers are bounded the same way
        for strategy in ("grid", "bitmap"):
            with pytest.raises(G.GcError) as e:
                G.generate(16, 3, "gray", strategy=strategy)
            assert e.value.code == 5, strategy
        # a batch: every job of the stuck group reports the timeout
        res = G.generate_batch([(12, 3, "lex", -1), (13, 4, "gray", -1)], ngroups=1)
        assert all(st.status == 5 for _, st in res)
    finally:
        del os.environ["GC_FAULT"]
    code = G.generate(15, 3, "lex").cpu().numpy().view(np.uint32)
    assert code.tolist() == oracle.greedy_pairwise(15, 3, "lex").tolist()
