"""Writes the oracle's codes for configurations too large for a test to
recompute, stored as size, SHA-256 of the little-endian uint32 list
(acceptance order), and the first and last words:
  --set large  tests/golden/large_expected.json: n = 31, d = 3 and n = 32,
               d = 4 in the four orders; n = 28, d = 5 lex
  --set batch  tests/golden/batch_expected.json: the 512 seeded instances of
               the batched workload (paper_1507_05398_gb300.workloads)
Calls only oracle/ (the exclusion-ball form O2, which equals the pairwise
definition wherever both run; the workload module only draws (n, d, order,
weight)).  Takes tens of CPU-minutes; run with

    python tests/golden/make_expected.py --set large [--jobs 8]
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
            "head": [int(x) for x in C[:8]], "last": int(C[-1]) if len(C) else None,
            "oracle_seconds": round(time.time() - t, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    ap.add_argument("--set", choices=["large", "batch"], default="large",
                    help="large: the n=28..32 sweeps; batch: the 512-instance batch")
    args = ap.parse_args()
    here = os.path.dirname(os.path.abspath(__file__))
    if args.set == "large":
        configs, out = CONFIGS, os.path.join(here, "large_expected.json")
    else:
        from paper_1507_05398_gb300.workloads import batch_instances
        configs, out = batch_instances(512, 1507), os.path.join(here, "batch_expected.json")
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        rows = pool.map(one, configs, chunksize=1)
    with open(out, "w") as f:
        json.dump({"generator": f"tests/golden/make_expected.py --set {args.set} (oracle O2)",
                   "codes": rows}, f, indent=1)
    print(f"wrote {out}: {len(rows)} codes")


if __name__ == "__main__":
    main()
