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


def _few_conflict_lists():
    """Lists for the bucketed resolver: runs of a code with stray vectors
    dropped in (the shape of a late window of a large sweep), random wide
    vectors with near copies, ragged sizes; then the shapes where it gives up
    (too many conflicts, too few varying bits, too many bucket pairs)."""
    out = []
    rng = np.random.default_rng(7)
    ham = oracle.greedy_ball(20, 3, "lex").astype(np.uint32)
    for size, stray, d in [(1000, 30, 3), (4096 - 64, 64, 3), (33, 2, 3), (31, 0, 2)]:
        run = ham[5000:5000 + size]
        extra = rng.integers(int(run[0]), int(run[-1]) + 1, stray, dtype=np.uint64)
        extra = np.setdiff1d(extra.astype(np.uint32), run)
        keys = np.concatenate([np.arange(len(run), dtype=float),
                               rng.uniform(0, len(run), len(extra))])
        lst = np.concatenate([run, extra])[np.argsort(keys, kind="stable")]
        out.append((f"hamming-run{size}+{len(extra)}", d, lst))
    for n_items, d in [(1, 4), (2, 8), (1000, 8), (4096, 8), (777, 6), (1500, 4)]:
        base = rng.integers(0, 1 << 32, n_items, dtype=np.uint64).astype(np.uint32)
        for i in rng.choice(n_items, n_items // 20, replace=False):
            flips = rng.choice(32, int(rng.integers(1, d + 1)), replace=False)
            base[i] = base[rng.integers(0, n_items)] ^ np.uint32(sum(1 << int(f) for f in flips))
        out.append((f"random32-{n_items}-d{d}", d, np.unique(base)[rng.permutation(len(np.unique(base)))]))
    out.append(("all12-d3", 3, rng.permutation(4096).astype(np.uint32)))
    out.append(("few-bits-d5", 5, (np.arange(8, dtype=np.uint32) * 3) | np.uint32(0xABC00000)))
    out.append(("8bits-d8", 8, rng.permutation(256).astype(np.uint32)))
    return out


@pytest.mark.parametrize("sparse", ["1", "0"])
@pytest.mark.parametrize("case", _few_conflict_lists(), ids=lambda c: c[0])
def test_resolve_few_conflicts(case, sparse, monkeypatch):
    _, d, lst = case
    monkeypatch.setenv("GC_SPARSE", sparse)
    want = oracle.resolve(d, lst)
    got = G().resolve(d, dev(lst)).cpu().numpy()
    assert got.tolist() == want.tolist()
