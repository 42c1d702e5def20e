"""Greedy codes over general B-orderings (Section 4.3) on the GPU."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def random_basis(n, rng):
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


def G():
    import paper_1507_05398_gb300 as g
    return g


@pytest.mark.parametrize("strategy", ["distance", "bitmap"])
def test_border_random_bases(strategy):
    rng = np.random.default_rng(1507)
    for n, d in [(8, 3), (10, 4), (12, 3), (14, 5), (16, 4), (18, 6), (20, 4)]:
        for _ in range(2):
            b = random_basis(n, rng)
            for w in (-1, n // 2):
                want = oracle.greedy_border(n, d, b, w)
                got = G().generate(n, d, b, w, strategy=strategy).cpu().numpy().view(np.uint32)
                assert got.tolist() == want.tolist(), (n, d, b, w)


def test_border_standard_and_gray_bases_equal_lex_and_gray():
    g = G()
    n, d = 20, 4
    std = [1 << j for j in range(n)]
    gray = [(1 << j) ^ (1 << (j - 1)) if j else 1 for j in range(n)]
    assert g.generate(n, d, std).cpu().tolist() == g.generate(n, d, "lex").cpu().tolist()
    assert g.generate(n, d, gray).cpu().tolist() == g.generate(n, d, "gray").cpu().tolist()


def test_border_dependent_basis_is_rejected():
    g = G()
    with pytest.raises(g.GcError) as e:
        g.generate(4, 2, [3, 5, 14, 8])
    assert e.value.code == 1
