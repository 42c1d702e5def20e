"""GPU parity of the Cartesian product of codes (Section 5, "Recursion in
Self orthogonal codes") with the oracle, including the paper's example and
the d = 8 range of its recursion figure (n = 15..26)."""
import numpy as np
import pytest

import oracle
import paper_1507_05398_gb300 as G

pytestmark = pytest.mark.gpu


def _dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=dtype))).cuda()


def _min_distance(words):
    w = np.asarray([int(v) for v in words], dtype=object)
    return min(bin(int(a) ^ int(b)).count("1") for i, a in enumerate(w) for b in w[:i])


@pytest.mark.parametrize("wide", [False, True])
def test_product_matches_oracle(wide):
    rng = np.random.default_rng(21)
    dt = np.int64 if wide else np.int32
    for la, lb, na, nb in [(8, 4, 16, 2), (13, 11, 300, 77), (5, 3, 1, 9), (20, 12, 1000, 1000)]:
        if not wide and la + lb > 32:
            continue
        A = rng.integers(0, 1 << la, na).astype(np.uint64)
        B = rng.integers(0, 1 << lb, nb).astype(np.uint64)
        got = G.product(_dev(A.astype(dt), dt), la, _dev(B.astype(dt), dt), lb).cpu().numpy()
        got = got.view(np.uint64) if wide else got.view(np.uint32).astype(np.uint64)
        assert got.tolist() == oracle.product64(A, B, la, lb).tolist()
    if wide:
        A = rng.integers(0, 1 << 40, 50).astype(np.uint64)
        B = rng.integers(0, 1 << 24, 60).astype(np.uint64)
        got = G.product(_dev(A.view(np.int64), np.int64), 40, _dev(B.view(np.int64), np.int64),
                        24).cpu().numpy().view(np.uint64)
        assert got.tolist() == oracle.product64(A, B, 40, 24).tolist()


def test_product_paper_example_code_12_4():
    P = G.selforth_product(12, 4, 4).cpu().numpy().view(np.uint32)
    A = oracle.greedy_selforth(8, 4, "lex")
    B = oracle.greedy_selforth(4, 4, "lex")
    assert B.tolist() == [0, 15]          # Code[4, 4] is the repetition code
    assert P.astype(np.uint64).tolist() == oracle.product64(A, B, 8, 4).tolist()
    assert len(P) == 32 and _min_distance(P) == 4


@pytest.mark.parametrize("n", range(15, 27))
def test_recursion_d8_range_of_the_figure(n):
    d, k = 8, 8
    P = G.selforth_product(n, d, k).cpu().numpy().view(np.uint32)
    A = oracle.greedy_selforth(n - k, d, "lex")
    B = oracle.greedy_selforth(k, d, "lex")
    assert P.astype(np.uint64).tolist() == oracle.product64(A, B, n - k, k).tolist()
    if len(P) > 1:
        assert _min_distance(P) >= d


def test_product_errors():
    a = _dev([1, 2], np.int32)
    with pytest.raises(G.GcError) as e:
        G.product(a, 20, a, 13)           # 33 bits in 32-bit words
    assert e.value.code == 1
    import torch
    with pytest.raises(G.GcError) as e:
        G.product(a, 4, a, 4, out=torch.empty(3, dtype=torch.int32, device="cuda"))
    assert e.value.code == 2
    with pytest.raises(TypeError):
        G.product(a, 4, _dev([1], np.int64), 4)
