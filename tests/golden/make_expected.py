"""Writes tests/golden/large_expected.json: the oracle's codes for the large
sweep configurations (n = 31, d = 3 and n = 32, d = 4 in the four orders;
n = 28, d = 5 lex), stored as size, SHA-256 of the little-endian uint32 list
(acceptance order), and the first and last words.  Calls only oracle/ (the
exclusion-ball form O2, which equals the pairwise definition wherever both
run).  Takes tens of CPU-minutes; run with

    python tests/golden/make_expected.py [--jobs 8]
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

CONFIGS = [(28, 5, "lex", -1)] + [(31, 3, o, -1) for o in ("lex", "gray", "grlex", "grevlex")] \
    + [(32, 4, o, -1) for o in ("lex", "gray", "grlex", "grevlex")]


def one(cfg):
    import oracle
    n, d, o, w = cfg
    t = time.time()
    C = oracle.greedy_ball(n, d, o, w)
    return {"n": n, "d": d, "ordering": o, "weight": w, "size": int(len(C)),
            "sha256": hashlib.sha256(C.astype("<u4").tobytes()).hexdigest(),
            "head": [int(x) for x in C[:8]], "last": int(C[-1]),
            "oracle_seconds": round(time.time() - t, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "large_expected.json"))
    args = ap.parse_args()
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        rows = pool.map(one, CONFIGS, chunksize=1)
    with open(args.out, "w") as f:
        json.dump({"generator": "tests/golden/make_expected.py (oracle O2)", "codes": rows}, f,
                  indent=1)
    print(json.dumps(rows, indent=1))


if __name__ == "__main__":
    main()
