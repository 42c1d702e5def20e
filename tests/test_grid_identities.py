"""Brute-force checks, on small n, of the facts the grid bitmap sweep rests
on (no GPU; the sweep itself is checked against the oracle by the GPU
tests):

- radius split: x lies within distance d-1 of c iff some v within distance
  d-2 of c lies within distance 1 of x (d >= 2), so marking radius-(d-2)
  balls and probing radius 1 finds exactly the covered candidates;
- survivor counters (d = 3): with cnt[v] the number of vectors of a set S
  within distance 1 of v, the sum of cnt over x's radius-1 ball is
  (n + 1) [x in S] + 2 |{y in S, y != x : d(x, y) <= 2}|, so a row meets
  another survivor within distance 2 iff its sum exceeds n + 1;
- stepping through a weight class: the next integer of the same weight
  (Gosper's rule) and the previous one (the complement's next one,
  complemented) walk the weight-k integers in order."""
import random

import pytest


def popc(v):
    return bin(v).count("1")


def ball(x, r, n):
    return [v for v in range(1 << n) if popc(v ^ x) <= r]


@pytest.mark.parametrize("n", [4, 5, 6])
@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_radius_split(n, d):
    for c in range(1 << n):
        marked = set(ball(c, d - 2, n))
        for x in range(1 << n):
            probe = any(popc(v ^ x) <= 1 for v in marked)
            assert probe == (popc(x ^ c) <= d - 1), (n, d, c, x)


@pytest.mark.parametrize("n", [5, 6, 7])
def test_survivor_counter_identity(n):
    rng = random.Random(1507 + n)
    for _ in range(20):
        S = set(rng.sample(range(1 << n), rng.randint(1, 1 << (n - 2))))
        cnt = [sum(1 for y in S if popc(v ^ y) <= 1) for v in range(1 << n)]
        for x in range(1 << n):
            total = sum(cnt[v] for v in ball(x, 1, n))
            near = sum(1 for y in S if y != x and popc(x ^ y) <= 2)
            assert total == (n + 1) * (x in S) + 2 * near
            if x in S:
                assert (total > n + 1) == (near > 0)


def next_same_weight(y):
    low = y & -y
    ripple = y + low
    return ripple | (((y ^ ripple) >> 2) >> (low.bit_length() - 1))


def prev_same_weight(y, n):
    mask = (1 << n) - 1
    return ~next_same_weight(~y & mask) & mask


@pytest.mark.parametrize("n", [1, 2, 5, 8, 12])
def test_stepping_through_a_weight_class(n):
    for k in range(0, n + 1):
        cls = sorted(v for v in range(1 << n) if popc(v) == k)
        for a, b in zip(cls, cls[1:]):
            assert next_same_weight(a) == b
            assert prev_same_weight(b, n) == a


def test_stepping_at_32_bits_stays_in_the_word():
    # the kernel's 32-bit words: the last step inside a class of n = 32
    # (the next-to-last weight-k integer to the last one, and back)
    for k in (1, 2, 16, 31):
        top = ((1 << k) - 1) << (32 - k)
        before = (((1 << (k - 1)) - 1) << (33 - k)) | (1 << (31 - k))
        assert popc(before) == k and before < top
        assert next_same_weight(before) == top < (1 << 32)
        assert prev_same_weight(top, 32) == before
