"""Parity of the whole CUDA sweep with the CPU oracle, element by element and
in acceptance order, through the C ABI (gc_generate_async / gc_generate)."""
import hashlib
import json
import os
from math import comb

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
ORDERS = ["lex", "gray", "grlex", "grevlex"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def G():
    import paper_1507_05398_gb300 as g
    return g


def gpu_code(n, d, o, w=-1, strategy=None, **kw):
    code, st = G().generate(n, d, o, w, strategy=strategy, return_stats=True, **kw)
    assert st.status == 0
    return code.cpu().numpy().view(np.uint32), st


@pytest.mark.parametrize("strategy", ["distance", "bitmap", "grid"])
@pytest.mark.parametrize("ordname", ORDERS)
def test_exhaustive_small(strategy, ordname):
    """Every n <= 10, every d in [0, n+1], with and without a weight."""
    for n in range(1, 11):
        for d in range(0, n + 2):
            for w in ([-1, n // 2, n] if n >= 2 else [-1, 0]):
                want = oracle.greedy_pairwise(n, d, ordname, w)
                got, st = gpu_code(n, d, ordname, w, strategy)
                assert got.tolist() == want.tolist(), (n, d, ordname, w, strategy)
                assert st.codewords == len(want)


@pytest.mark.parametrize("strategy", ["distance", "bitmap"])
def test_config_hamming_15(strategy):
    """n = 15, d = 3, lex: the [15,11,3] Hamming code, 2048 words, XOR-closed."""
    got, st = gpu_code(15, 3, "lex", -1, strategy)
    assert got.tolist() == oracle.greedy_pairwise(15, 3, "lex").tolist()
    assert len(got) == 2048
    s = set(got.tolist())
    assert all((int(a) ^ int(b)) in s for a in got[:64] for b in got)


def test_config_golay_24():
    """n = 24, d = 8, lex: extended Golay, 4096 words (the benchmark's first
    code, in the benchmark's launch configuration)."""
    got, st = gpu_code(24, 8, "lex")
    want, pos = oracle.greedy_ball(24, 8, "lex", with_pos=True)
    assert got.tolist() == want.tolist()
    assert st.dense_tests == oracle.dense_tests(pos, 1 << 24)


@pytest.mark.parametrize("ordname", ORDERS)
def test_config_n20_d4(ordname):
    """n = 20, d = 4 in the four orders (the rest of the benchmark workload)."""
    got, st = gpu_code(20, 4, ordname)
    want, pos = oracle.greedy_ball(20, 4, ordname, with_pos=True)
    assert got.tolist() == want.tolist()
    assert len(got) == 16384
    assert st.dense_tests == oracle.dense_tests(pos, 1 << 20)


@pytest.mark.parametrize("strategy", ["distance", "bitmap", "grid"])
@pytest.mark.parametrize("ordname", ORDERS)
@pytest.mark.parametrize("n,d", [(16, 3), (17, 5), (18, 4), (19, 6), (21, 3)])
def test_mid_sizes(strategy, ordname, n, d):
    """Many windows, ragged tiles, survivor truncation."""
    want = oracle.greedy_ball(n, d, ordname)
    got, _ = gpu_code(n, d, ordname, -1, strategy)
    assert got.tolist() == want.tolist()


@pytest.mark.parametrize("strategy", ["distance", "bitmap", "grid"])
@pytest.mark.parametrize("ordname", ORDERS)
@pytest.mark.parametrize("n,d,w", [(16, 4, 5), (18, 6, 6), (20, 4, 3), (14, 3, 7), (22, 6, 4)])
def test_constant_weight(strategy, ordname, n, d, w):
    want = oracle.greedy_pairwise(n, d, ordname, w)
    got, _ = gpu_code(n, d, ordname, w, strategy)
    assert got.tolist() == want.tolist()
    assert all(bin(int(x)).count("1") == w for x in got)


@pytest.mark.parametrize("strategy", ["distance", "bitmap", "grid"])
def test_small_windows_and_degenerate(strategy):
    """Tiny windows force thousands of window steps; d = 2 keeps half the
    space (survivors beyond the resolver's capacity every window)."""
    for n, d, o in [(16, 2, "lex"), (14, 2, "grevlex"), (18, 2, "gray")]:
        want = oracle.greedy_ball(n, d, o)
        got, _ = gpu_code(n, d, o, -1, strategy)
        assert got.tolist() == want.tolist()
    want = oracle.greedy_ball(18, 5, "grlex")
    got, _ = gpu_code(18, 5, "grlex", -1, strategy, window_min=32, window_max=64,
                      survivor_target=8)
    assert got.tolist() == want.tolist()


def test_capacity_and_host_entry():
    g = G()
    want = oracle.greedy_pairwise(15, 3, "gray")
    assert g.generate_host(15, 3, "gray").tolist() == want.tolist()
    with pytest.raises(g.GcError) as e:
        g.generate_host(15, 3, "gray", capacity=100)
    assert e.value.code == 2
    code = g.generate(15, 3, "gray", capacity=100)
    assert code.cpu().numpy().view(np.uint32).tolist() == want[:100].tolist()


def _large():
    p = os.path.join(GOLDEN, "large_expected.json")
    if not os.path.exists(p):
        return []
    return json.load(open(p))["codes"]


@pytest.mark.parametrize("row", _large(), ids=lambda r: f"n{r['n']}d{r['d']}{r['ordering']}")
def test_large_configs_against_stored_oracle(row):
    """n = 31, d = 3 and n = 32, d = 4 (all orders), n = 28, d = 5 lex:
    compared with the oracle's stored list digest, plus closed forms."""
    n, d, o, w = row["n"], row["d"], row["ordering"], row["weight"]
    strategies = ["grid", "bitmap", "distance"] if n == 28 else [None, "bitmap"]
    for strategy in strategies:
        got, st = gpu_code(n, d, o, w, strategy)
        assert len(got) == row["size"]
        assert got[:8].tolist() == row["head"] and int(got[-1]) == row["last"]
        assert hashlib.sha256(got.astype("<u4").tobytes()).hexdigest() == row["sha256"]
    if (n, d, o) == (31, 3, "lex"):
        assert len(got) == 2 ** 26 and np.all(np.diff(got.astype(np.int64)) > 0)


def test_n32_d4_lex_is_the_parity_extension_of_n31_d3_lex():
    """At full size, the GPU's n = 32, d = 4 lex code is its n = 31, d = 3 lex
    code with an overall parity bit appended, word for word."""
    a, _ = gpu_code(31, 3, "lex")
    b, _ = gpu_code(32, 4, "lex")
    par = a.copy()
    for sh in (16, 8, 4, 2, 1):
        par ^= par >> np.uint32(sh)
    ext = (a.astype(np.uint64) << np.uint64(1)) | (par & np.uint32(1)).astype(np.uint64)
    assert len(a) == len(b) == 2 ** 26
    assert np.array_equal(ext, b.astype(np.uint64))


def test_large_bitmap_sweeps_plan_the_grid_strategy():
    """A bitmap problem of 2^26 or more candidates is planned for the grid
    strategy (every SM in every window); smaller ones keep the pipelined
    bitmap sweep, which a batch or a server also runs for grid jobs."""
    g = G()
    assert g.plan(31, 3, "lex").strategy == g.STRATEGY_BITMAP_GRID
    assert g.plan(32, 4, "grevlex").strategy == g.STRATEGY_BITMAP_GRID
    assert g.plan(20, 4, "lex").strategy == g.STRATEGY_BITMAP
    code, st = gpu_code(26, 3, "gray")
    assert st.strategy == g.STRATEGY_BITMAP_GRID
    assert code.tolist() == oracle.greedy_ball(26, 3, "gray").tolist()
    res = g.generate_batch([(26, 3, "gray", -1, "grid"), (12, 3, "lex", -1)])
    assert res[0][1].strategy == g.STRATEGY_BITMAP and res[0][0].tolist() == code.tolist()


@pytest.mark.parametrize("o", ORDERS)
@pytest.mark.parametrize("n,d,w", [(22, 3, -1), (23, 4, -1), (24, 5, -1), (22, 4, 9), (24, 3, 11)])
def test_grid_strategy_mid_and_weighted(o, n, d, w):
    """The grid strategy on codes of many windows, with and without a weight
    (windows cut at 4096 survivors, pair lists, conflict-matrix fallbacks)."""
    got, st = gpu_code(n, d, o, w, "grid")
    want = oracle.greedy_ball(n, d, o, w)
    assert got.tolist() == want.tolist()
    assert st.strategy == G().STRATEGY_BITMAP_GRID and st.codewords == len(want)


@pytest.mark.parametrize("env", [{"GC_GRID_PROBE": "0"}, {"GC_GRID_PROBE": "1"},
                                 {"GC_GRID_EARLY": "1"}, {"GC_GRID_EARLY": "0"},
                                 {"GC_GRID_CONF": "0"}])
def test_grid_radius_split_both_ways(env, monkeypatch):
    """The grid sweep either marks radius-(d-1) balls and looks up one bit,
    or marks radius-(d-2) balls and probes the candidate's radius-1
    neighbourhood; with early marks, window t-1's balls go into the bitmap
    before window t's rows are probed against it instead of tested against
    window t-1's accepts; for d = 3, byte counters of the window's survivors
    let only the rows that meet another survivor run the pair tests.
    GC_GRID_PROBE / GC_GRID_EARLY / GC_GRID_CONF force each form.  All give
    the oracle's code, in every order, with and without a weight."""
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    for n, d, o, w in [(18, 3, "lex", -1), (19, 4, "gray", -1), (20, 4, "grevlex", -1),
                       (20, 5, "grlex", -1), (21, 6, "lex", -1), (18, 4, "grevlex", 7),
                       (20, 4, "gray", 9), (9, 4, "lex", -1), (5, 3, "grlex", -1),
                       (20, 3, "grevlex", -1), (19, 3, "gray", 6), (4, 2, "lex", -1),
                       (21, 3, "lex", -1), (3, 3, "gray", -1), (2, 3, "lex", -1)]:
        got, st = gpu_code(n, d, o, w, "grid")
        assert got.tolist() == oracle.greedy_ball(n, d, o, w).tolist(), (env, n, d, o, w)


@pytest.mark.parametrize("cap", ["1", "40", "700"])
def test_grid_long_pair_lists_from_l2(cap, monkeypatch):
    """Windows whose pair list exceeds what shared memory takes run their
    first rounds over the list in L2, then carry on in shared memory;
    GC_GRID_PAIR_SMEM lowers that limit so small codes take the path."""
    monkeypatch.setenv("GC_GRID_PAIR_SMEM", cap)
    for n, d, o, w in [(20, 3, "lex", -1), (21, 3, "gray", -1), (20, 4, "grlex", -1),
                       (20, 3, "grevlex", -1), (19, 5, "lex", -1), (18, 3, "grlex", 6)]:
        got, st = gpu_code(n, d, o, w, "grid")
        assert got.tolist() == oracle.greedy_ball(n, d, o, w).tolist(), (cap, n, d, o, w)
        assert st.pair_windows > 0


@pytest.mark.parametrize("early", ["0", "1"])
def test_grid_strategy_on_fewer_ctas(early, monkeypatch):
    """The grid strategy on a grid of 1, 2 and 7 CTAs (many rows per CTA),
    with window t-1's balls marked during the tests or before the rows."""
    monkeypatch.setenv("GC_GRID_EARLY", early)
    for n, d, o in [(20, 4, "grlex"), (19, 3, "lex")]:
        want = oracle.greedy_ball(n, d, o)
        for grid in (1, 2, 7):
            got, _ = gpu_code(n, d, o, -1, "grid", grid=grid)
            assert got.tolist() == want.tolist(), (n, d, o, grid)


# (n, d, order, strategy, survivor target, whether pair lists must decide
# some window of a whole-GPU launch)
PAIR_CASES = [
    (20, 3, "lex", "bitmap", 2048, True),
    (22, 3, "grlex", "bitmap", 1024, True),
    (23, 7, "lex", "bitmap", 1024, True),
    (19, 4, "grlex", "bitmap", 1024, False),
    (16, 2, "gray", "bitmap", 1024, False),
    (20, 3, "gray", "distance", 2048, False),
]


@pytest.mark.parametrize("case", PAIR_CASES, ids=lambda c: f"n{c[0]}d{c[1]}{c[2]}-{c[3]}")
def test_generator_pair_lists(case, monkeypatch):
    """Pipelined bitmap jobs in a large group decide a window from the list
    of its conflicting pairs that the generator CTAs found, after a window
    that accepted at least 7/8 of its survivors (GC_PAIRS=0 turns it off,
    GC_PAIRS=2 lists every window's pairs).
    The code is the oracle's either way, and on the codes with such windows
    the pair lists decide some of them."""
    n, d, o, strategy, target, expect = case
    want = oracle.greedy_ball(n, d, o)
    for pairs in ("1", "0", "2"):
        monkeypatch.setenv("GC_PAIRS", pairs)
        got, st = gpu_code(n, d, o, -1, strategy, survivor_target=target)
        assert got.tolist() == want.tolist(), pairs
        if pairs == "0" or strategy == "distance":
            assert st.pair_windows == 0 and st.pair_fallbacks == 0
        elif pairs == "2" or expect:
            # GC_PAIRS=2: every window after the first goes through the lists
            assert st.pair_windows > 0


@pytest.mark.parametrize("mode", [("1", "1"), ("1", "0"), ("0", "1")],
                         ids=["whole-window", "whole-window-tail", "blocked"])
@pytest.mark.parametrize("o", ORDERS)
def test_whole_window_matrices(o, mode, monkeypatch):
    """n = 20, d = 4 bitmap codes on the whole GPU: a pipelined window of more
    survivors than one conflict matrix takes is decided from the whole
    window's conflict matrix, which the generator CTAs build, and is cut
    after as many survivors as that matrix holds.  GC_DENSE_CUT=0 keeps the
    windows whole and sends the survivors beyond the matrix to the blocked
    matrices; GC_DENSE=0 uses the blocked matrices only.  The code is the
    oracle's in every mode."""
    dense, cut = mode
    monkeypatch.setenv("GC_DENSE", dense)
    monkeypatch.setenv("GC_DENSE_CUT", cut)
    got, st = gpu_code(20, 4, o, -1, "bitmap")
    assert got.tolist() == oracle.greedy_ball(20, 4, o).tolist(), (o, mode)
    assert st.codewords == len(got)


def test_pair_list_overflow_falls_back_to_matrices(monkeypatch):
    """GC_PAIRS=2 on n = 20, d = 4 grevlex (windows with thousands of
    conflicting pairs): some windows are decided from the lists, the rest
    overflow them and go to the conflict matrices; the code is the oracle's."""
    monkeypatch.setenv("GC_PAIRS", "2")
    got, st = gpu_code(20, 4, "grevlex", -1, "bitmap")
    assert got.tolist() == oracle.greedy_ball(20, 4, "grevlex").tolist()
    assert st.pair_windows > 0 and st.pair_fallbacks > 0
