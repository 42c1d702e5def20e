"""Self-orthogonal greedy codes (Section 4.4) on the GPU against the oracle."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
ORDERS = ["lex", "gray", "grlex", "grevlex"]


def G():
    import paper_1507_05398_gb300 as g
    return g


def gpu(n, d, o, w=-1, **kw):
    code, st = G().generate(n, d, o, w, constraint="self_orthogonal", return_stats=True, **kw)
    assert st.status == 0
    return code.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("ordname", ORDERS)
def test_selforth_exhaustive_small(ordname):
    for n in range(1, 11):
        for d in range(0, n + 2):
            for w in ([-1, n // 2] if n >= 2 else [-1]):
                want = oracle.greedy_selforth(n, d, ordname, w)
                assert gpu(n, d, ordname, w).tolist() == want.tolist(), (n, d, ordname, w)


def test_selforth_golay_codes():
    """Section 7: extended Golay [24,12,8] and the [22,11,6] code."""
    for n, d, size in ((24, 8, 4096), (22, 6, 2048)):
        got = gpu(n, d, "lex")
        assert len(got) == size
        assert got.tolist() == oracle.greedy_selforth(n, d, "lex").tolist()


@pytest.mark.parametrize("ordname", ORDERS)
@pytest.mark.parametrize("n,d", [(16, 4), (18, 6), (20, 4), (21, 5)])
def test_selforth_mid_sizes(ordname, n, d):
    assert gpu(n, d, ordname).tolist() == oracle.greedy_selforth(n, d, ordname).tolist()


def test_selforth_in_a_batch_and_forced_bitmap_request():
    g = G()
    probs = [(16, 4, "lex", -1, None, "self_orthogonal"), (16, 4, "lex", -1),
             (14, 4, "gray", 6, "bitmap", "self_orthogonal"), (18, 6, "grlex", -1, None, "self_orthogonal")]
    res = g.generate_batch(probs)
    for p, (code, st) in zip(probs, res):
        n, d, o, w = p[:4]
        so = len(p) > 5
        want = oracle.greedy_selforth(n, d, o, w) if so else oracle.greedy_ball(n, d, o, w)
        assert code.tolist() == want.tolist(), p
