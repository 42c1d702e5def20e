"""GPU parity of the wide sweep (uint64 words, n <= 64) with the oracle's
64-bit forms: element-by-element equality of the code in acceptance order,
the statistics, the closed forms that hold at any size, the equivalence with
the narrow sweep where the lengths overlap, and the argument edges."""
from math import comb

import numpy as np
import pytest

import oracle
import paper_1507_05398_gb300 as G

pytestmark = pytest.mark.gpu
ORDERS = ["lex", "gray", "grlex", "grevlex"]


def as_u64(t):
    return t.cpu().numpy().view(np.uint64)


def blocks(n, w):
    return [((1 << w) - 1) << (w * k) for k in range(n // w)]


@pytest.mark.parametrize("ordname", ORDERS)
@pytest.mark.parametrize("n,w,d", [(33, 2, 3), (35, 3, 4), (35, 5, 6), (40, 4, 6), (48, 3, 4),
                                   (64, 2, 3), (64, 3, 4), (34, 5, 4)])
def test_wide_constant_weight_parity(ordname, n, w, d):
    want, pos = oracle.greedy64(n, d, ordname, w, with_pos=True)
    code, st = G.generate64(n, d, ordname, w, return_stats=True)
    got = as_u64(code)
    assert got.tolist() == want.tolist()
    assert st.codewords == len(want)
    assert st.status == 0 and st.strategy == G.STRATEGY_DISTANCE
    if ordname != "gray":  # no skipped ranks: the dense count is exact
        assert st.dense_tests == oracle.dense_tests(pos, comb(n, w))


@pytest.mark.parametrize("ordname", ["lex", "grlex", "grevlex"])
def test_wide_one_million_candidates(ordname):
    # C(35, 6) = 1,623,160 candidates, several hundred windows
    n, w, d = 35, 6, 8
    want = oracle.greedy64(n, d, ordname, w)
    got = as_u64(G.generate64(n, d, ordname, w))
    assert got.tolist() == want.tolist()


@pytest.mark.parametrize("ordname", ORDERS)
@pytest.mark.parametrize("n,w,d", [(34, 4, 4), (36, 2, 2), (40, 6, 8)])
def test_wide_self_orthogonal_parity(ordname, n, w, d):
    want = oracle.greedy64(n, d, ordname, w, orth=True)
    got = as_u64(G.generate64(n, d, ordname, w, constraint="self_orthogonal"))
    assert got.tolist() == want.tolist()


@pytest.mark.parametrize("ordname", ORDERS)
@pytest.mark.parametrize("n,d,w", [(20, 4, -1), (16, 5, -1), (12, 3, 5), (24, 8, -1), (18, 6, 6)])
def test_wide_equals_narrow_for_short_codes(ordname, n, d, w):
    narrow = G.generate(n, d, ordname, w).cpu().numpy().view(np.uint32)
    wide = as_u64(G.generate64(n, d, ordname, w))
    assert wide.tolist() == narrow.astype(np.uint64).tolist()


@pytest.mark.parametrize("ordname", ORDERS)
def test_wide_full_space_d_equals_n(ordname):
    # 2^33 ranks; with d = n only 0 and the all-ones vector are at distance n
    n = 33
    code, st = G.generate64(n, n, ordname, -1, return_stats=True)
    assert as_u64(code).tolist() == [0, (1 << n) - 1]
    assert st.candidates == 1 << n


@pytest.mark.parametrize("n,w", [(34, 3), (64, 5), (57, 4)])
def test_wide_gray_weight_rank_space(n, w):
    # Gray with a weight sweeps only the C(n, w) weight-w vectors, in Gray
    # order (closed-form unrank); d = 2w forces disjoint supports
    code, st = G.generate64(n, 2 * w, "gray", w, return_stats=True)
    assert as_u64(code).tolist() == blocks(n, w)
    assert st.candidates == comb(n, w)
    if comb(n, w) < 2_000_000:
        assert as_u64(code).tolist() == oracle.greedy64(n, 2 * w, "gray", w).tolist()


def test_wide_edges_and_host_entry():
    assert as_u64(G.generate64(64, 5, "lex", 0)).tolist() == [0]
    assert as_u64(G.generate64(64, 5, "grevlex", 64)).tolist() == [(1 << 64) - 1]
    seq = oracle.order_list64(33, "grevlex", 2)
    assert as_u64(G.generate64(33, 1, "grevlex", 2)).tolist() == seq.tolist()   # d <= 1
    assert as_u64(G.generate64(33, 40, "grevlex", 2)).tolist() == seq[:1].tolist()  # d > n
    # the synchronous entry with a host buffer, and its capacity protocol
    want = oracle.greedy64(40, 6, "lex", 4)
    assert G.generate64_host(40, 6, "lex", 4).tolist() == want.tolist()
    with pytest.raises(G.GcError) as e:
        G.generate64_host(40, 6, "lex", 4, capacity=3)
    assert e.value.code == 2
    with pytest.raises(G.GcError):
        G.generate64(40, 6, "lex", 4, strategy="bitmap")   # no wide bitmap
    # generate() routes n > 32 to the wide entry
    assert as_u64(G.generate(40, 6, "lex", 4)).tolist() == want.tolist()
