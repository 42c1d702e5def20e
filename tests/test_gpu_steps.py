"""Parity of each CUDA step, called through the C ABI, with the oracle's
step forms."""
from math import comb

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
ORDERS = ["lex", "gray", "grlex", "grevlex"]


def G():
    import paper_1507_05398_gb300 as g
    return g


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint32)).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("ordname", ORDERS)
def test_unrank_and_rank(ordname):
    g = G()
    for n in list(range(1, 13)) + [16, 20]:
        seq = oracle.order_list(n, ordname)
        got = host(g.unrank(n, ordname, -1, 0, len(seq)))
        assert got.tolist() == seq.tolist(), n
        r = g.rank(n, ordname, dev(seq)).cpu().numpy()
        assert r.tolist() == list(range(len(seq)))
        # a window in the middle
        a = len(seq) // 3
        b = min(len(seq), a + 77)
        assert host(g.unrank(n, ordname, -1, a, b - a)).tolist() == seq[a:b].tolist()
        for w in (0, n // 2, n):
            sub = oracle.order_list(n, ordname, w)
            assert host(g.unrank(n, ordname, w, 0, len(sub))).tolist() == sub.tolist()


def test_unrank_large_n_spot():
    g = G()
    for ordname in ORDERS:
        for n in (28, 31, 32):
            N = 1 << n
            ranks = [0, 1, 2, N // 3, N // 2, N - 2, N - 1]
            for r in ranks:
                v = int(host(g.unrank(n, ordname, -1, r, 1))[0])
                assert int(g.rank(n, ordname, dev([v])).cpu()[0]) == r


@pytest.mark.parametrize("n,d,nc,nk", [(10, 3, 100, 7), (20, 5, 5000, 300), (24, 8, 9000, 20000),
                                       (32, 6, 4097, 33), (16, 4, 1, 0), (16, 4, 0, 10)])
def test_block_test(n, d, nc, nk):
    rng = np.random.default_rng(n * 100 + d)
    cand = rng.integers(0, 1 << n, nc, dtype=np.uint64).astype(np.uint32)
    code = rng.integers(0, 1 << n, nk, dtype=np.uint64).astype(np.uint32)
    want = oracle.block_test(d, cand, code)
    got = G().block_test(d, dev(cand), dev(code)).cpu().numpy()
    assert got.tolist() == want.tolist()


@pytest.mark.parametrize("n,d,nc", [(12, 3, 4096), (20, 4, 1000), (16, 6, 257), (9, 2, 300),
                                    (24, 8, 4000), (10, 1, 100)])
def test_resolve(n, d, nc):
    rng = np.random.default_rng(nc)
    cand = np.unique(rng.integers(0, 1 << n, nc, dtype=np.uint64)).astype(np.uint32)
    rng.shuffle(cand)
    want = oracle.resolve(d, cand)
    got = G().resolve(d, dev(cand)).cpu().numpy()
    assert got.tolist() == want.tolist()


@pytest.mark.parametrize("n,d", [(3, 2), (5, 3), (8, 9), (12, 4), (20, 3), (18, 7)])
def test_bitmap_mark(n, d):
    rng = np.random.default_rng(n + d)
    code = rng.integers(0, 1 << n, 50, dtype=np.uint64).astype(np.uint32)
    want = oracle.ball_mark(n, d, code)
    got = host(G().bitmap_mark(n, d, dev(code)))
    assert got.tolist() == want.tolist()


@pytest.mark.parametrize("ordname", ORDERS)
def test_bitmap_scan(ordname):
    g = G()
    rng = np.random.default_rng(5)
    for n, w in [(9, -1), (16, -1), (16, 5), (20, 8)]:
        N = (1 << n) if w < 0 else comb(n, w)
        bm = (rng.integers(0, 1 << 32, max(1, (1 << n) // 32), dtype=np.uint64)
              & rng.integers(0, 1 << 32, max(1, (1 << n) // 32), dtype=np.uint64)).astype(np.uint32)
        for r0, cnt in [(0, N), (N // 5, N // 3), (N - 1, 1), (7, 0)]:
            want = oracle.scan(n, ordname, w, bm, r0, cnt)
            got, found = g.bitmap_scan(n, ordname, w, dev(bm), r0, cnt)
            assert found == len(want)
            assert host(got).tolist() == want.tolist()
