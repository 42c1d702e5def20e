"""Pins for the oracle's 64-bit forms (vectors of up to 64 coordinates; the
constant-weight codes of Section 7 go to length 35).  Each check ties them to
something other than themselves: the independently pinned 32-bit forms where
the lengths overlap, the closed form of constant-weight codes whose distance
forces disjoint supports, the prefix structure of the lex, Gray and grlex
orders, and the O3 characterisation; the Cartesian product of codes (Section
5) by the example the paper gives and by brute force."""
from math import comb

import numpy as np
import pytest

import oracle

ORDERS = ["lex", "gray", "grlex", "grevlex"]


def blocks(n, w):
    """The disjoint-support code: weight-w blocks of consecutive coordinates,
    starting at the last coordinate (the lowest bits)."""
    return [((1 << w) - 1) << (w * k) for k in range(n // w)]


@pytest.mark.parametrize("ordname", ORDERS)
def test_order64_equals_32bit_definitions(ordname):
    for n in range(1, 11):
        for w in sorted({-1, 0, n // 2, n}):
            a = oracle.order_list64(n, ordname, w)
            b = oracle.order_sorted(n, ordname, w)
            assert a.astype(np.int64).tolist() == b.astype(np.int64).tolist(), (n, w)


@pytest.mark.parametrize("ordname", ORDERS)
def test_greedy64_equals_32bit_oracle(ordname):
    for n in range(1, 12):
        for d in range(0, n + 2):
            for w in ([-1, n // 2] if n >= 2 else [-1]):
                a, pa = oracle.greedy64(n, d, ordname, w, with_pos=True)
                b, pb = oracle.greedy_pairwise(n, d, ordname, w, with_pos=True)
                assert a.astype(np.int64).tolist() == b.astype(np.int64).tolist(), (n, d, w)
                assert pa.tolist() == pb.tolist()


@pytest.mark.parametrize("ordname", ORDERS)
def test_greedy64_selforth_equals_32bit_oracle(ordname):
    for n in range(2, 12):
        for d in (2, 3, 4, 6):
            for w in (-1, 2 * (n // 4)):
                a = oracle.greedy64(n, d, ordname, w, orth=True)
                b = oracle.greedy_selforth(n, d, ordname, w)
                assert a.astype(np.int64).tolist() == b.astype(np.int64).tolist(), (n, d, w)


@pytest.mark.parametrize("ordname", ORDERS)
@pytest.mark.parametrize("n,w", [(33, 1), (33, 2), (35, 3), (35, 5), (40, 4), (47, 3),
                                 (64, 1), (64, 2), (64, 3)])
def test_disjoint_blocks_closed_form(ordname, n, w):
    # two weight-w words are at distance >= 2w only with disjoint supports,
    # and all distances between them are even, so d = 2w-1 acts as 2w
    want = blocks(n, w)
    for d in (2 * w - 1, 2 * w):
        got = [int(v) for v in oracle.greedy64(n, d, ordname, w)]
        assert got == want, (n, w, d)
    if w % 2 == 0:  # disjoint even-weight blocks are also self-orthogonal
        got = [int(v) for v in oracle.greedy64(n, 2 * w, ordname, w, orth=True)]
        assert got == want


@pytest.mark.parametrize("ordname", ["lex", "gray", "grlex"])
@pytest.mark.parametrize("n,m,w,d", [(40, 20, 3, 4), (36, 16, 4, 4), (33, 18, 2, 3)])
def test_prefix_is_the_shorter_code(ordname, n, m, w, d):
    # in lex, Gray and grlex order the weight-w vectors below 2^m come first,
    # in the m-bit order; so the code's words below 2^m are the m-bit code
    C = [int(v) for v in oracle.greedy64(n, d, ordname, w)]
    low = [v for v in C if v < (1 << m)]
    assert C[:len(low)] == low
    assert low == oracle.greedy_pairwise(m, d, ordname, w).astype(np.int64).tolist()


@pytest.mark.parametrize("ordname", ORDERS)
def test_verify64_accepts_greedy_rejects_perturbed(ordname):
    n, d, w = 36, 4, 3
    C = oracle.greedy64(n, d, ordname, w)
    assert len(C) > 10
    assert oracle.verify64(n, d, ordname, w, C) == 0
    assert oracle.verify64(n, d, ordname, w, C[:-1]) != 0          # not maximal
    assert oracle.verify64(n, d, ordname, w, C[::-1]) != 0         # out of order
    bad = C.copy(); bad[4] ^= np.uint64(3)
    assert oracle.verify64(n, d, ordname, w, bad) != 0
    assert oracle.verify64(n, d, ordname, w, np.append(C, C[2])) != 0


def test_degenerate_64():
    assert oracle.greedy64(64, 5, "lex", 0).tolist() == [0]
    assert [int(v) for v in oracle.greedy64(64, 5, "grevlex", 64)] == [2 ** 64 - 1]
    with pytest.raises(RuntimeError):
        oracle.greedy64(64, 5, "lex", -1)   # 2^64 candidates: needs a weight
    assert oracle.candidate_count64(64, 32) == comb(64, 32)
    assert oracle.candidate_count64(40, -1) == 2 ** 40
    for ordname in ORDERS:
        seq = oracle.order_list64(34, ordname, 2)
        assert len(seq) == comb(34, 2)
        assert oracle.greedy64(34, 1, ordname, 2).tolist() == seq.tolist()   # d <= 1: all
        assert oracle.greedy64(34, 40, ordname, 2).tolist() == seq[:1].tolist()  # d > n: first


# ---------------------------------------------------------------- products
def _min_distance(words):
    w = [int(v) for v in words]
    return min(bin(a ^ b).count("1") for i, a in enumerate(w) for b in w[:i])


def _self_orthogonal(words):
    w = [int(v) for v in words]
    return all(bin(a).count("1") % 2 == 0 for a in w) and \
        all(bin(a & b).count("1") % 2 == 0 for i, a in enumerate(w) for b in w[:i])


def test_product_example_of_section5():
    # the self-orthogonal greedy [8, 4] code combined with Code[4, 4] (the
    # repetition code of length 4) gives a length-12 code of distance 4
    A = oracle.greedy_selforth(8, 4, "lex")
    assert len(A) == 16
    B = [0, 0b1111]
    P = oracle.product64(A, B, 8, 4)
    assert len(P) == 32
    assert all(int(v) < (1 << 12) for v in P)
    assert _min_distance(P) == 4
    assert _self_orthogonal(P)
    # linear: the span has dimension 4 + 1
    assert set(int(a) ^ int(b) for a in P for b in P) == set(int(v) for v in P)
    # order: A outermost, B inner
    assert [int(v) for v in P[:2]] == [int(A[0]) << 4, (int(A[0]) << 4) | 15]


def test_product_distance_is_the_smaller_one_bruteforce():
    rng = np.random.default_rng(3)
    for _ in range(20):
        la, lb = int(rng.integers(3, 9)), int(rng.integers(3, 9))
        A = np.unique(rng.integers(0, 1 << la, int(rng.integers(2, 8)))).astype(np.uint64)
        B = np.unique(rng.integers(0, 1 << lb, int(rng.integers(2, 8)))).astype(np.uint64)
        if len(A) < 2 or len(B) < 2:
            continue
        P = oracle.product64(A, B, la, lb)
        assert len(P) == len(A) * len(B)
        assert _min_distance(P) == min(_min_distance(A), _min_distance(B))
    with pytest.raises(RuntimeError):
        oracle.product64([1], [1], 40, 30)
