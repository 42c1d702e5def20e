"""Seeded random differential tests of the whole sweep against the oracle.
Problem parameters (n, d, order, weight, constraint) and launch parameters
(strategy, CTA count, survivor target, window bounds) are drawn together, so
the launch shapes the planner never picks (one CTA, windows of one rank,
survivor targets far off) are exercised as well as the usual ones."""
import numpy as np
import pytest

import oracle
import paper_1507_05398_gb300 as G

pytestmark = pytest.mark.gpu
ORDERS = ["lex", "gray", "grlex", "grevlex"]


def _cases(seed, count, wide):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        n = int(rng.integers(20, 41)) if wide else int(rng.integers(4, 19))
        d = int(rng.integers(0, min(n, 12) + 2))
        o = ORDERS[int(rng.integers(0, 4))]
        if wide:
            w = int(rng.integers(1, 5))
            if oracle.candidate_count64(n, w) > 200_000:
                continue
        else:
            w = -1 if rng.random() < 0.6 else int(rng.integers(0, n + 1))
        orth = bool(rng.random() < 0.2)
        strategy = "distance" if (wide or orth or rng.random() < 0.5) else "bitmap"
        grid = int(rng.choice([1, 2, 3, 7, 19, 152]))
        target = int(rng.choice([1, 8, 64, 512, 4096]))
        wmin = int(rng.choice([1, 32, 256]))
        wmax = int(rng.choice([0, 64, 4096]))
        if wmax and wmax < wmin:
            wmax = wmin
        out.append((n, d, o, w, orth, strategy, grid, target, wmin, wmax))
    return out


def _id(c):
    n, d, o, w, orth, st, grid, target, wmin, wmax = c
    return f"n{n}d{d}{o}w{w}{'o' if orth else ''}-{st[0]}-g{grid}t{target}w{wmin}-{wmax}"


def _plan(case):
    n, d, o, w, orth, strategy, grid, target, wmin, wmax = case
    kw = dict(strategy=strategy, grid=grid, survivor_target=target, window_min=wmin,
              constraint="self_orthogonal" if orth else None)
    if wmax:
        kw["window_max"] = wmax
    return kw


@pytest.mark.parametrize("case", _cases(1507, 120, False), ids=_id)
def test_random_problem_and_launch_shape(case):
    n, d, o, w, orth = case[:5]
    want = oracle.greedy_selforth(n, d, o, w) if orth else oracle.greedy_ball(n, d, o, w)
    code, st = G.generate(n, d, o, w, return_stats=True, **_plan(case))
    assert st.status == 0
    assert code.cpu().numpy().view(np.uint32).tolist() == want.tolist()


@pytest.mark.parametrize("case", _cases(2015, 40, True), ids=_id)
def test_random_wide_problem_and_launch_shape(case):
    n, d, o, w, orth = case[:5]
    want = oracle.greedy64(n, d, o, w, orth=orth)
    code, st = G.generate64(n, d, o, w, return_stats=True, **_plan(case))
    assert st.status == 0
    assert code.cpu().numpy().view(np.uint64).tolist() == want.tolist()
