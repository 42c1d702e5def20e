"""Pins for the CPU oracle: each check ties it to something other than itself
(the paper's worked example, closed forms of the codes Section 7 names,
textbook order definitions, brute force over all subsets on tiny inputs)."""
import itertools
import os
from math import comb

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ORDERS = ["lex", "gray", "grlex", "grevlex"]


def popc(x: int) -> int:
    return bin(int(x)).count("1")


def xor_closed(words) -> bool:
    s = set(int(x) for x in words)
    return all((a ^ b) in s for a in s for b in s)


def weight_dist(words):
    out = {}
    for x in words:
        k = popc(x)
        out[k] = out.get(k, 0) + 1
    return out


# ---------------------------------------------------------------- Example 1
def test_example1_worked_steps():
    """Example 1 (Section 4.1): n = 3, d = 2, lex -> {000, 011, 101, 110}."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "example1_n3_d2_lex.txt"))
             if l.strip() and not l.startswith("#")]
    n, d, ordname = int(lines[0][0]), int(lines[0][1]), lines[0][2]
    accepted = [(s, int(v)) for s, v in (l for l in lines[1:] if len(l) == 2)]
    rejected = [l for l in lines[1:] if len(l) == 3]
    for s, v in accepted:
        assert int(s, 2) == v  # coordinate 1 is the most significant bit
    got = oracle.greedy_pairwise(n, d, ordname)
    assert got.tolist() == [v for _, v in accepted]
    # each rejected vector is within d-1 of one of the codewords it met
    for _, vec, against in rejected:
        x = int(vec, 2)
        assert any(popc(x ^ int(c, 2)) < d for c in against.split(","))


# ---------------------------------------------------------------- orderings
def reflected_gray(n):
    """Binary-reflected Gray code by its recursive construction."""
    seq = ["0", "1"]
    for _ in range(n - 1):
        seq = ["0" + s for s in seq] + ["1" + s for s in reversed(seq)]
    return [int(s, 2) for s in seq]


@pytest.mark.parametrize("n", range(1, 11))
def test_gray_matches_reflected_construction(n):
    g = oracle.order_list(n, "gray")
    assert g.tolist() == reflected_gray(n)
    assert all(popc(int(a) ^ int(b)) == 1 for a, b in zip(g[:-1], g[1:]))


@pytest.mark.parametrize("n", range(1, 11))
@pytest.mark.parametrize("ordname", ORDERS)
def test_stream_order_equals_comparator_sort(n, ordname):
    for w in [-1] + list(range(0, n + 1)):
        a = oracle.order_list(n, ordname, w)
        b = oracle.order_sorted(n, ordname, w)
        assert a.tolist() == b.tolist(), (n, ordname, w)
        assert len(a) == (2 ** n if w < 0 else comb(n, w))
        assert len(set(a.tolist())) == len(a)


def test_graded_orders_by_hand():
    """Textbook graded orders on 3 variables (x1 = most significant bit)."""
    # grlex ascending: 1 < x3 < x2 < x1 < x2x3 < x1x3 < x1x2 < x1x2x3
    assert oracle.order_list(3, "grlex").tolist() == [0, 1, 2, 4, 3, 5, 6, 7]
    # grevlex ascending, 4 variables, degree 2: the last variable decides
    # x3x4 < x2x4 < x1x4 < x2x3 < x1x3 < x1x2
    want = [0b0011, 0b0101, 0b1001, 0b0110, 0b1010, 0b1100]
    assert oracle.order_list(4, "grevlex", 2).tolist() == want
    assert oracle.order_list(4, "grlex", 2).tolist() == sorted(want)


@pytest.mark.parametrize("n", [5, 8, 12])
def test_grevlex_pairwise_rule(n):
    seq = oracle.order_list(n, "grevlex")
    for a, b in zip(seq[:-1], seq[1:]):
        a, b = int(a), int(b)
        if popc(a) != popc(b):
            assert popc(a) < popc(b)
        else:
            low = (a ^ b) & -(a ^ b)
            assert a & low


# ---------------------------------------------------------------- brute force
def greedy_characterised(n, d, seq):
    """All subsets of the candidate list that are (1) pairwise >= d and (2)
    cover every other candidate by an earlier member within d-1."""
    found = []
    N = len(seq)
    for mask in range(1 << N):
        members = [i for i in range(N) if mask >> i & 1]
        ok = all(popc(seq[i] ^ seq[j]) >= d for i, j in itertools.combinations(members, 2))
        if not ok:
            continue
        ok = all(any(j < i and popc(seq[i] ^ seq[j]) <= d - 1 for j in members)
                 for i in range(N) if not mask >> i & 1)
        if ok:
            found.append([seq[i] for i in members])
    return found


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("ordname", ORDERS)
def test_bruteforce_unique_characterisation(n, ordname):
    for w in [-1] + list(range(n + 1)):
        seq = [int(x) for x in oracle.order_sorted(n, ordname, w)]
        if len(seq) > 16:
            continue
        for d in range(0, n + 2):
            found = greedy_characterised(n, d, seq)
            assert len(found) == 1, (n, ordname, w, d, found)
            assert oracle.greedy_pairwise(n, d, ordname, w).tolist() == found[0]
            assert oracle.greedy_ball(n, d, ordname, w).tolist() == found[0]


# ---------------------------------------------------------------- closed forms
def _fixture_codes():
    rows = []
    for l in open(os.path.join(GOLDEN, "perfect_codes.txt")):
        if l.strip() and not l.startswith("#"):
            f = l.split()
            wd = {int(k): int(v) for k, v in (t.split(":") for t in f[4:])}
            rows.append((int(f[0]), int(f[1]), f[2], int(f[3]), wd))
    return rows


@pytest.mark.parametrize("row", _fixture_codes(), ids=lambda r: f"n{r[0]}d{r[1]}")
def test_named_codes(row):
    """Section 7: Hamming (n = 7, 15), Golay [23,12,7], extended Golay [24,12,8]."""
    n, d, ordname, size, wd = row
    C = oracle.greedy_ball(n, d, ordname)
    assert len(C) == size
    assert weight_dist(C) == wd
    assert xor_closed(C) if size <= 4096 else True
    assert C[0] == 0


@pytest.mark.parametrize("m", [2, 3, 4])
def test_hamming_perfect(m):
    n = 2 ** m - 1
    C = oracle.greedy_pairwise(n, 3, "lex")
    assert len(C) == 2 ** (n - m)
    assert len(C) * (n + 1) == 2 ** n  # radius-1 balls tile the space
    assert xor_closed(C)
    assert min(popc(x) for x in C[1:]) == 3
    assert weight_dist(C).get(3, 0) == n * (n - 1) // 6


def test_golay_perfect():
    C = oracle.greedy_ball(23, 7, "lex")
    vol = sum(comb(23, i) for i in range(4))
    assert len(C) * vol == 2 ** 23


@pytest.mark.slow
@pytest.mark.skipif(not os.environ.get("GC_SLOW"), reason="minutes of CPU; set GC_SLOW=1")
def test_hamming_31_closed_form():
    """[31,26,3] Hamming code: 2^26 words (perfect), XOR-closed (sampled)."""
    C = oracle.greedy_ball(31, 3, "lex")
    assert len(C) == 2 ** 26
    rng = np.random.default_rng(1507)
    s = set(C.tolist())
    a = C[rng.integers(0, len(C), 2000)]
    b = C[rng.integers(0, len(C), 2000)]
    assert all(int(x ^ y) in s for x, y in zip(a, b))


# ---------------------------------------------------------------- relations
@pytest.mark.parametrize("n,d", [(6, 3), (9, 3), (10, 4), (11, 5), (13, 4), (14, 6)])
@pytest.mark.parametrize("ordname", ["lex", "gray"])
def test_b_ordering_codes_are_linear(n, d, ordname):
    """Lex and Gray are B-orderings; B-greedy codes are linear (the Brualdi-
    Pless result Section 4.3 cites), so |C| is a power of two and C is
    closed under XOR."""
    C = oracle.greedy_pairwise(n, d, ordname)
    assert len(C) & (len(C) - 1) == 0
    assert xor_closed(C)


@pytest.mark.parametrize("n,d", [(12, 4), (16, 4), (16, 8)])
def test_lex_and_grlex_same_words_for_power_of_two_d(n, d):
    """Section 7: for d a power of two the lex and graded-lex greedy codes
    have the same words (a conjecture the paper observed up to n = 30)."""
    assert set(oracle.greedy_ball(n, d, "lex").tolist()) == \
        set(oracle.greedy_ball(n, d, "grlex").tolist())


@pytest.mark.parametrize("n,d", [(7, 3), (11, 5), (15, 3)])
def test_parity_extension(n, d):
    """Lexicode (n+1, d+1) is lexicode (n, d) with an overall parity bit
    appended (odd d); observed relation, consistent with Golay -> extended."""
    a = oracle.greedy_pairwise(n, d, "lex")
    b = oracle.greedy_pairwise(n + 1, d + 1, "lex")
    ext = [(int(x) << 1) | (popc(x) & 1) for x in a]
    assert ext == b.tolist()


def _parity_ext(v: int) -> int:
    return (v << 1) | (popc(v) & 1)


def _large_rows():
    import json
    p = os.path.join(os.path.dirname(__file__), "golden", "large_expected.json")
    return {(r["n"], r["d"], r["ordering"]): r for r in json.load(open(p))["codes"]}


def test_parity_extension_relates_the_stored_n31_and_n32_codes():
    """The stored n = 32, d = 4 lex code is the n = 31, d = 3 lex code with an
    overall parity bit appended (the relation test_parity_extension checks
    at n = 7, 11, 15): same size, and the stored first and last words map
    onto each other."""
    rows = _large_rows()
    a, b = rows[(31, 3, "lex")], rows[(32, 4, "lex")]
    assert a["size"] == b["size"] == 2 ** 26
    assert [_parity_ext(x) for x in a["head"]] == b["head"]
    assert _parity_ext(a["last"]) == b["last"]


def _hamming_syndrome(x, first_bit=0):
    """Syndrome of the binary Hamming code whose parity check maps bit i of
    the vector (value 2^i) to the column i + 1 (numpy, elementwise)."""
    s = np.zeros_like(x)
    for i in range(32):
        bit = (x >> np.uint32(i)) & np.uint32(1)
        s ^= bit * np.uint32(first_bit + i + 1)
    return s


def test_hamming_lexicode_closed_form_at_small_n():
    """The d = 3 lexicode of length 2^m - 1 is the Hamming code with the
    parity check i -> i + 1 (Section 7 names the perfect codes): checked
    against the oracle at n = 3, 7, 15."""
    for n in (3, 7, 15):
        x = np.arange(1 << n, dtype=np.uint32)
        closed = x[_hamming_syndrome(x) == 0]
        assert closed.tolist() == oracle.greedy_ball(n, 3, "lex").tolist(), n


def test_stored_n31_and_n32_digests_from_the_hamming_closed_form():
    """The stored n = 31, d = 3 lex digest (oracle O2) is the Hamming
    [31,26,3] code of the closed form above, in increasing order, and the
    stored n = 32, d = 4 lex digest is that code with an overall parity bit
    appended (extended Hamming [32,26,4]).  The code is built in increasing
    order without a sort: a word is (hi << 16) | lo, and for each high part
    the low parts are the 2048 whose syndrome cancels the high part's."""
    import hashlib
    rows = _large_rows()
    lo = np.arange(1 << 16, dtype=np.uint32)
    syn_lo = _hamming_syndrome(lo)
    by_syn = [lo[syn_lo == v] for v in range(32)]
    assert all(len(b) == 2048 for b in by_syn)
    table = np.stack(by_syn)                                  # [32][2048], increasing
    h31, h32 = hashlib.sha256(), hashlib.sha256()
    size = 0
    for h0 in range(0, 1 << 15, 4096):
        hi = np.arange(h0, h0 + 4096, dtype=np.uint32)
        syn_hi = _hamming_syndrome(hi, first_bit=16)
        words = ((hi[:, None] << np.uint32(16)) | table[syn_hi]).reshape(-1)
        h31.update(words.astype("<u4").tobytes())
        par = words.copy()
        for sh in (16, 8, 4, 2, 1):
            par ^= par >> np.uint32(sh)
        ext = (words << np.uint32(1)) | (par & np.uint32(1))   # < 2^32: bit 31 of words is 0
        h32.update(ext.astype("<u4").tobytes())
        size += words.size
    assert size == rows[(31, 3, "lex")]["size"] == rows[(32, 4, "lex")]["size"] == 1 << 26
    assert h31.hexdigest() == rows[(31, 3, "lex")]["sha256"]
    assert h32.hexdigest() == rows[(32, 4, "lex")]["sha256"]


@pytest.mark.skipif(not os.environ.get("GC_SLOW"), reason="a minute of CPU; set GC_SLOW=1")
def test_parity_extension_of_the_n31_oracle_code_gives_the_stored_n32_digest():
    """The whole n = 31, d = 3 lex code from the oracle, extended by parity,
    hashes to the stored n = 32, d = 4 lex digest (extended Hamming
    [32,26,4]), which make_expected.py wrote from the n = 32 sweep."""
    import hashlib
    a = oracle.greedy_ball(31, 3, "lex").astype(np.uint32)
    par = a.copy()
    for sh in (16, 8, 4, 2, 1):
        par ^= par >> np.uint32(sh)
    ext = (a.astype(np.uint64) << np.uint64(1)) | (par & np.uint32(1)).astype(np.uint64)
    assert ext.max() < 2 ** 32
    digest = hashlib.sha256(ext.astype("<u4").tobytes()).hexdigest()
    assert digest == _large_rows()[(32, 4, "lex")]["sha256"]


# ---------------------------------------------------------------- edge cases
@pytest.mark.parametrize("ordname", ORDERS)
def test_degenerate_distances(ordname):
    n = 9
    seq = oracle.order_list(n, ordname)
    for d in (0, 1):
        assert oracle.greedy_pairwise(n, d, ordname).tolist() == seq.tolist()
    with pytest.raises(RuntimeError):
        oracle.greedy_pairwise(n, -1, ordname)
    for d in (n + 1, n + 5):
        assert oracle.greedy_pairwise(n, d, ordname).tolist() == [0]
    # d = n: only 0 and the all-ones vector
    assert oracle.greedy_pairwise(n, n, ordname).tolist() == [0, 2 ** n - 1]


@pytest.mark.parametrize("ordname", ORDERS)
@pytest.mark.parametrize("n,w", [(10, 2), (12, 3), (12, 4), (13, 5)])
def test_constant_weight_closed_forms(ordname, n, w):
    C = oracle.greedy_pairwise(n, 2 * w, ordname, w)
    assert len(C) == n // w  # disjoint supports
    assert all(popc(x) == w for x in C)
    allw = oracle.greedy_pairwise(n, 2, ordname, w)
    assert len(allw) == comb(n, w)
    assert oracle.greedy_pairwise(n, 3, ordname, w).tolist() == \
        oracle.greedy_pairwise(n, 4, ordname, w).tolist()  # distances are even
    assert oracle.greedy_pairwise(n, 5, ordname, 0).tolist() == [0]
    assert oracle.greedy_pairwise(n, 5, ordname, n).tolist() == [2 ** n - 1]


def test_constant_weight_lex_equals_grlex():
    for n, d, w in [(12, 4, 3), (14, 6, 5), (16, 4, 4)]:
        assert oracle.greedy_pairwise(n, d, "lex", w).tolist() == \
            oracle.greedy_pairwise(n, d, "grlex", w).tolist()


# ---------------------------------------------------------------- O1 = O2, O3
@pytest.mark.parametrize("ordname", ORDERS)
def test_pairwise_equals_ball(ordname):
    for n in range(1, 13):
        for d in range(0, n + 2):
            for w in ([-1, n // 2] if n >= 2 else [-1]):
                a = oracle.greedy_pairwise(n, d, ordname, w, with_pos=True)
                b = oracle.greedy_ball(n, d, ordname, w, with_pos=True)
                assert a[0].tolist() == b[0].tolist(), (n, d, ordname, w)
                assert a[1].tolist() == b[1].tolist()


@pytest.mark.parametrize("ordname", ORDERS)
def test_pairwise_equals_ball_n20(ordname):
    assert oracle.greedy_pairwise(16, 4, ordname).tolist() == \
        oracle.greedy_ball(16, 4, ordname).tolist()
    assert oracle.greedy_pairwise(16, 5, ordname).tolist() == \
        oracle.greedy_ball(16, 5, ordname).tolist()


def test_verify_accepts_greedy_rejects_perturbed():
    for ordname in ORDERS:
        C = oracle.greedy_pairwise(10, 3, ordname)
        assert oracle.verify(10, 3, ordname, -1, C) == 0
        assert oracle.verify(10, 3, ordname, -1, C[:-1]) != 0      # not maximal
        assert oracle.verify(10, 3, ordname, -1, C[::-1]) != 0     # out of order
        bad = C.copy(); bad[5] ^= 1
        assert oracle.verify(10, 3, ordname, -1, bad) != 0
        assert oracle.verify(10, 3, ordname, -1, np.append(C, C[3] ^ 1)) != 0


def test_dense_tests_count():
    # every candidate accepted: candidate i meets i codewords
    _, pos = oracle.greedy_pairwise(8, 1, "lex", with_pos=True)
    assert oracle.dense_tests(pos, 256) == 256 * 255 // 2
    # direct count on a small case
    C, pos = oracle.greedy_pairwise(7, 3, "gray", with_pos=True)
    seq = oracle.order_list(7, "gray")
    direct = sum(int((pos < i).sum()) for i in range(len(seq)))
    assert oracle.dense_tests(pos, len(seq)) == direct


# ---------------------------------------------------------------- step forms
def test_step_block_test_bruteforce():
    rng = np.random.default_rng(7)
    for n, d in [(6, 2), (9, 3), (12, 5), (20, 6)]:
        cand = rng.integers(0, 1 << n, 300, dtype=np.uint64).astype(np.uint32)
        code = rng.integers(0, 1 << n, 40, dtype=np.uint64).astype(np.uint32)
        want = [int(all(popc(int(x) ^ int(c)) >= d for c in code)) for x in cand]
        assert oracle.block_test(d, cand, code).tolist() == want
    assert oracle.block_test(3, [5], []).tolist() == [1]


@pytest.mark.parametrize("ordname", ORDERS)
def test_step_resolve_over_whole_order_is_greedy(ordname):
    for n, d, w in [(9, 3, -1), (11, 4, -1), (12, 4, 5), (8, 5, -1)]:
        seq = oracle.order_list(n, ordname, w)
        idx = oracle.resolve(d, seq)
        assert seq[idx].tolist() == oracle.greedy_pairwise(n, d, ordname, w).tolist()


def test_step_ball_mark_covers_space_and_matches_bruteforce():
    for n, d in [(7, 3), (10, 4), (12, 5)]:
        C = oracle.greedy_pairwise(n, d, "lex")
        bm = oracle.ball_mark(n, d, C)
        # maximality of the greedy code: every vector within d-1 of a codeword
        assert all((int(bm[v >> 5]) >> (v & 31)) & 1 for v in range(1 << n))
    rng = np.random.default_rng(3)
    code = rng.integers(0, 1 << 9, 5, dtype=np.uint64).astype(np.uint32)
    bm = oracle.ball_mark(9, 3, code)
    for v in range(1 << 9):
        want = any(popc(v ^ int(c)) <= 2 for c in code)
        assert bool((int(bm[v >> 5]) >> (v & 31)) & 1) == want


@pytest.mark.parametrize("ordname", ORDERS)
def test_step_scan(ordname):
    n = 9
    empty = np.zeros(16, dtype=np.uint32)
    assert oracle.scan(n, ordname, -1, empty, 0, 512).tolist() == \
        oracle.order_list(n, ordname).tolist()
    assert oracle.scan(n, ordname, -1, empty, 100, 50).tolist() == \
        oracle.order_list(n, ordname)[100:150].tolist()
    full = np.full(16, 0xFFFFFFFF, dtype=np.uint32)
    assert len(oracle.scan(n, ordname, -1, full, 0, 512)) == 0
    rng = np.random.default_rng(11)
    bm = rng.integers(0, 1 << 32, 16, dtype=np.uint64).astype(np.uint32)
    seq = oracle.order_list(n, ordname)
    want = [int(x) for x in seq[37:400] if not (int(bm[x >> 5]) >> (int(x) & 31)) & 1]
    assert oracle.scan(n, ordname, -1, bm, 37, 363).tolist() == want
    # weight-restricted rank spaces: rank i is the i-th weight-w vector of the
    # full order
    w = 4
    sub = [int(x) for x in seq if popc(x) == w]
    assert sub == oracle.order_list(n, ordname, w).tolist()
    assert oracle.scan(n, ordname, w, empty, 0, comb(n, w)).tolist() == sub
    sw = [x for x in sub[20:90] if not (int(bm[x >> 5]) >> (x & 31)) & 1]
    assert oracle.scan(n, ordname, w, bm, 20, 70).tolist() == sw


# ---------------------------------------------------------------- self-orthogonal
def test_selforth_extended_and_baby_golay():
    """Section 7: greedy self-orthogonal generation gives the extended Golay
    code [24,12,8]; the baby Golay [22,11,6] (also named there) at n=22, d=6."""
    rows = {(r[0], r[1]): r for r in _fixture_codes()}
    C = oracle.greedy_selforth(24, 8, "lex")
    assert len(C) == 4096 and weight_dist(C) == rows[(24, 8)][4]
    B = oracle.greedy_selforth(22, 6, "lex")
    assert len(B) == 2 ** 11
    assert min(popc(x) for x in B[1:]) == 6
    for code, n in ((C, 24), (B, 22)):  # self-dual: linear, self-orthogonal, 2^(n/2) words
        assert xor_closed(code)
        assert all(popc(int(a) & int(b)) % 2 == 0 for a in code[:40] for b in code)


def test_selforth_extended_hamming_8():
    C = oracle.greedy_selforth(8, 4, "lex")
    assert len(C) == 16 and weight_dist(C) == {0: 1, 4: 14, 8: 1}


def _selforth_characterised(n, d, seq):
    found = []
    N = len(seq)
    for mask in range(1 << N):
        members = [i for i in range(N) if mask >> i & 1]
        if any(popc(seq[i]) % 2 for i in members):
            continue
        if any(popc(seq[i] ^ seq[j]) < d or popc(seq[i] & seq[j]) % 2
               for i, j in itertools.combinations(members, 2)):
            continue
        ok = all(popc(seq[i]) % 2 or any(j < i and (popc(seq[i] ^ seq[j]) < d or
                                                     popc(seq[i] & seq[j]) % 2)
                                          for j in members)
                 for i in range(N) if not mask >> i & 1)
        if ok:
            found.append([seq[i] for i in members])
    return found


@pytest.mark.parametrize("ordname", ORDERS)
def test_selforth_bruteforce(ordname):
    for n in (2, 3, 4):
        seq = [int(x) for x in oracle.order_sorted(n, ordname)]
        for d in range(0, n + 2):
            found = _selforth_characterised(n, d, seq)
            assert len(found) == 1
            assert oracle.greedy_selforth(n, d, ordname).tolist() == found[0]


# ---------------------------------------------------------------- B-orderings
def random_basis(n, rng):
    """An invertible n x n matrix over F_2 (rows = basis vectors), drawn by
    rejection."""
    while True:
        rows = [int(v) for v in rng.integers(0, 1 << n, n, dtype=np.uint64)]
        m, rank = list(rows), 0
        for bit in range(n - 1, -1, -1):
            piv = next((j for j in range(rank, n) if m[j] >> bit & 1), None)
            if piv is None:
                continue
            m[rank], m[piv] = m[piv], m[rank]
            for j in range(n):
                if j != rank and m[j] >> bit & 1:
                    m[j] ^= m[rank]
            rank += 1
        if rank == n:
            return rows


def test_border_sequence_definition():
    """Section 4.3: {0, b1, b2, b2+b1, b3, b3+b1, b3+b2, b3+b2+b1, b4, ...}."""
    b = [0b0011, 0b0101, 0b1110, 0b0001]
    seq = [oracle.border_vector(4, b, r) for r in range(16)]
    assert seq[:9] == [0, b[0], b[1], b[1] ^ b[0], b[2], b[2] ^ b[0], b[2] ^ b[1],
                       b[2] ^ b[1] ^ b[0], b[3]]
    assert sorted(seq) == list(range(16))


@pytest.mark.parametrize("n,d", [(8, 3), (10, 4), (12, 5), (13, 3)])
def test_border_standard_and_gray_bases(n, d):
    std = [1 << j for j in range(n)]
    gray = [(1 << j) ^ (1 << (j - 1)) if j else 1 for j in range(n)]
    assert oracle.greedy_border(n, d, std).tolist() == oracle.greedy_pairwise(n, d, "lex").tolist()
    assert oracle.greedy_border(n, d, gray).tolist() == oracle.greedy_pairwise(n, d, "gray").tolist()


@pytest.mark.parametrize("n,d", [(9, 3), (11, 4), (12, 6)])
def test_border_codes_are_linear(n, d):
    rng = np.random.default_rng(n * 10 + d)
    for _ in range(3):
        C = oracle.greedy_border(n, d, random_basis(n, rng))
        assert len(C) & (len(C) - 1) == 0
        assert xor_closed(C)


def test_border_bruteforce_and_dependent_basis():
    rng = np.random.default_rng(3)
    for n in (2, 3, 4):
        b = random_basis(n, rng)
        seq = [oracle.border_vector(n, b, r) for r in range(1 << n)]
        for d in range(0, n + 2):
            found = greedy_characterised(n, d, seq)
            assert len(found) == 1
            assert oracle.greedy_border(n, d, b).tolist() == found[0]
    with pytest.raises(RuntimeError):
        oracle.greedy_border(4, 2, [1, 2, 3, 8])
