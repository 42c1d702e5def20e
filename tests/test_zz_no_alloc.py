"""gc_generate_noalloc, the allocation-free entry point for callers that
cannot call cudaMalloc (runtimes without a device allocator, device memory
owned by another framework's pool, latency-critical paths): through the C ABI
its output must equal the oracle's code and the regular gc_generate_async
output, element for element, on two calls in a row (the static scratch is
shared and keeps the previous call's contents).  Kept in a file of its own,
collected last."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

CASES = [(15, 3, "lex", -1, None), (20, 4, "gray", -1, "bitmap"), (18, 5, "grevlex", -1, "distance"),
         (16, 4, "grlex", 6, None), (24, 8, "lex", -1, None)]


def test_noalloc_matches_regular_entry_point_twice():
    import torch

    import paper_1507_05398_gb300 as G

    assert G.noalloc_scratch_bytes() == 32 << 20
    for n, d, o, w, strategy in CASES:
        want = G.generate(n, d, o, w, strategy=strategy).cpu().numpy().view(np.uint32)
        # the regular entry point agrees with the oracle (pins both paths)
        assert want.tolist() == oracle.greedy_ball(n, d, o, w).tolist(), (n, d, o, w)
        cap = G.capacity_bound(n, d, w)
        for _ in range(2):
            out = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
            st = torch.zeros(ctypes.sizeof(G.Stats), dtype=torch.uint8, device="cuda")
            G.generate_noalloc(n, d, o, w, out=out, stats=st, strategy=strategy)
            s = G.stats_from(st)
            assert s.status == 0
            got = out[:s.codewords].cpu().numpy().view(np.uint32)
            assert got.tolist() == want.tolist(), (n, d, o, w, strategy)


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch

    import paper_1507_05398_gb300 as G

    out = torch.empty(16, dtype=torch.int32, device="cuda")
    st = torch.zeros(ctypes.sizeof(G.Stats), dtype=torch.uint8, device="cuda")
    with pytest.raises(G.GcError) as e:  # a 2^30-bit exclusion map does not fit
        G.generate_noalloc(30, 3, "lex", out=out, stats=st, strategy="bitmap")
    assert e.value.code == 6 and "static scratch" in str(e.value)
    with pytest.raises(G.GcError) as e:  # an invalid problem is GC_ERR_INVALID
        G.generate_noalloc(33, 3, "lex", out=out, stats=st)
    assert e.value.code == 1
