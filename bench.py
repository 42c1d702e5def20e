"""Benchmark of the ordered greedy code sweep on one GB300 (or N replicas).

Workload (one "step"): the five codes n=24, d=8 lex (extended Golay) and
n=20, d=4 in lex, Gray, graded-lex and graded-reverse-lex order, each one
whole sweep over all 2^n candidates.  Metric: candidate-codeword distance
tests per second, counted as dense-equivalent tests (for each candidate, the
number of codewords accepted before it -- the tests a sweep without early
exit performs, the paper's naive kernel) divided by the device time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs the same
workload as an independent replica (the sweep of one code does not shard).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = [(24, 8, "lex"), (20, 4, "lex"), (20, 4, "gray"), (20, 4, "grlex"), (20, 4, "grevlex")]
WORKLOAD_NAME = "n=24 d=8 lex + n=20 d=4 x {lex, gray, grlex, grevlex}"
METRIC = "candidate-codeword distance tests/s (dense-equivalent)"
L2_FLUSH_BYTES = 256 << 20


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms.  Entering
    waits for the first sample (so sampling is running when the timed region
    starts); leaving waits for one sample after the region ends.  summary()
    covers the samples from the region's start to that one."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self._got.append((time.monotonic(), line))

    def _wait_for(self, pred, timeout):
        end = time.monotonic() + timeout
        while time.monotonic() < end and not pred():
            time.sleep(0.005)

    def __enter__(self):
        import threading
        self._got, self.lines = [], []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._reader = threading.Thread(target=self._read, daemon=True)
            self._reader.start()
            self._wait_for(lambda: self._got, 5.0)
        except Exception:
            self.proc = None
        self.t0 = time.monotonic()
        return self

    def __exit__(self, *exc):
        t1 = time.monotonic()
        if self.proc is not None:
            self._wait_for(lambda: self._got and self._got[-1][0] > t1, 1.0)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self._reader.join(timeout=2)
            after = [ts for ts, _ in self._got if ts > t1]
            t_end = after[0] if after else t1
            # the last sample before the region, those inside it, the first after
            before = [ts for ts, _ in self._got if ts <= self.t0]
            t_beg = before[-1] if before else self.t0
            self.lines = [l for ts, l in self._got if t_beg <= ts <= t_end]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ reference
def run_reference(args):
    """The CPU oracle, single-threaded, as it stands: each step is one code of
    the workload (rotating), so K steps cover a bounded sample of it."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    dense = 0
    seconds = 0.0
    sample = []
    for i in range(args.warmup + args.steps):
        n, d, o = WORKLOAD[i % len(WORKLOAD)]
        t = time.perf_counter()
        C, pos = oracle.greedy_pairwise(n, d, o, with_pos=True)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            dense += oracle.dense_tests(pos, 1 << n)
            seconds += dt
            sample.append(f"n={n} d={d} {o}")
    value = dense / seconds
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "tests/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * seconds / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (fully determined by n, d, order)",
        "config": {"workload": WORKLOAD_NAME, "parallelism": "host, 1 thread"},
        "cpu_baseline": {"value": value, "unit": "tests/s", "cores": 1, "kind": "oracle",
                         "sample": "; ".join(sample) + " (pairwise oracle, one code per step)",
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "tests/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours
def cpu_baseline_sample():
    import oracle
    oracle.build()
    dense, secs, parts = 0, 0.0, []
    for n, d, o in [(24, 8, "lex"), (20, 4, "lex")]:
        t = time.perf_counter()
        C, pos = oracle.greedy_pairwise(n, d, o, with_pos=True)
        secs += time.perf_counter() - t
        dense += oracle.dense_tests(pos, 1 << n)
        parts.append(f"n={n} d={d} {o}")
    return {"value": dense / secs, "unit": "tests/s", "cores": 1, "kind": "oracle",
            "sample": " + ".join(parts) + " (pairwise oracle, whole sweeps, "
                      f"{secs:.1f} s)", "cpu": cpu_model()}


def _code_only(text: str) -> str:
    """C/C++ source with comments removed and whitespace runs collapsed
    (string and character literals kept as written)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash() -> str:
    """Hash of the CUDA/C++ sources' code (comments and layout ignored): the
    recorded DRAM traffic stays valid across comment-only edits."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_1507_05398_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))
                   + glob.glob(os.path.join(csrc, "*.h")))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        h.update(_code_only(open(f, encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of the batched sweep from the committed ncu
    summary, or None if the kernel sources changed since that capture."""
    p = os.path.join(ROOT, "profiles", "sweep_kernel_bench_workload_traffic.md")
    try:
        txt = open(p).read()
    except OSError:
        return None
    vals = dict(l.split(":", 1) for l in txt.splitlines()
                if l.startswith(("traffic_bytes_per_launch:", "kernel_source_sha256_16:")))
    if vals.get("kernel_source_sha256_16", "").strip() != kernel_source_hash():
        return None
    return int(vals["traffic_bytes_per_launch"].strip())


def run_ours(args):
    import numpy as np
    import torch

    global WORKLOAD, WORKLOAD_NAME
    if args.only:
        n, d, o = args.only.split(",")
        WORKLOAD = [(int(n), int(d), o)]
        WORKLOAD_NAME = f"n={n} d={d} {o} (single code)"

    import paper_1507_05398_gb300 as G

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    probs = [(n, d, o, -1) for n, d, o in WORKLOAD]
    ngroups = len(probs) if args.groups is None else args.groups

    # resident buffers: the whole workload as one prepared batch, one
    # persistent launch per step, replayed from a CUDA graph
    batch = G.BatchBuffers(probs, ngroups=ngroups)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    batch.launch(stream)
    torch.cuda.synchronize()
    try:
        graph = batch.capture()
        step = graph.replay
        launch_kind = "CUDA graph replay of one batched persistent launch"
    except Exception as e:  # capture refused: launch directly
        print(f"bench: CUDA graph capture failed ({e}); launching directly", file=sys.stderr)
        step = lambda: batch.launch(stream)  # noqa: E731
        launch_kind = "one batched persistent launch"
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    results = batch.results()
    for (code, st), p in zip(results, probs):
        if st.status != 0:
            raise RuntimeError(f"sweep failed for {p}: {st.as_dict()}")
    dense = sum(st.dense_tests for _, st in results)
    executed = sum(st.executed_tests for _, st in results)
    launches_per_step = 1  # the sweep; ball tables were built when the batch was prepared

    # timed region: K steps, L2 flushed before each, CUDA events per step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.fill_(s & 0xff)
            ev[s][0].record(stream)
            step()
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    mean_step_ms = statistics.mean(step_ms)
    if world > 1:
        t = torch.tensor([mean_step_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        mean_step_ms = float(t.item())
    value = world * dense / (mean_step_ms * 1e-3)
    stats_now = [st for _, st in batch.results()]

    # the same codes one launch each (gc_generate_async), for comparison
    singles = []
    for n, d, o, w in probs:
        cap = G.capacity_bound(n, d, w)
        ws_bytes = G.workspace_size(n, d, o, w)
        ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
        base = (-ws.data_ptr()) % 256
        singles.append((n, d, o, w, torch.empty(cap, dtype=torch.int32, device=dev),
                        torch.zeros(ctypes.sizeof(G.Stats), dtype=torch.uint8, device=dev),
                        ws[base:base + ws_bytes]))
    per_code_ms = {}
    for n, d, o, w, out, st, ws in singles:
        G.generate_async(n, d, o, w, out=out, stats=st, workspace=ws, stream=stream)
        times = []
        for s in range(args.steps):
            flush.fill_(s & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            G.generate_async(n, d, o, w, out=out, stats=st, workspace=ws, stream=stream)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        per_code_ms[f"n={n} d={d} {o}"] = statistics.mean(times)
    single_ms = sum(per_code_ms.values())

    # end to end through the public API: generate_batch launches the batch
    # (prepared on the first, untimed, call and kept), waits and copies the
    # statistics and every output to the host in one transfer
    e2e_times, d2h = [], G.batch_result_bytes(probs)
    for s in range(0 if args.no_e2e else args.warmup + args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = G.generate_batch(probs, ngroups=ngroups)
        if s >= args.warmup:
            e2e_times.append(time.perf_counter() - t)
        for (code, st), p in zip(res, probs):
            if st.status != 0 or len(code) != st.codewords:
                raise RuntimeError(f"end-to-end sweep failed for {p}: {st.as_dict()}")
    e2e_value = world * dense / statistics.mean(e2e_times) if e2e_times else None

    # roofline of the sweep kernel: executed distance tests per second against
    # the measured register-operand test rate of this GPU
    peak, _ = G.probe_test_rate()
    achieved = executed / (mean_step_ms * 1e-3)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = cpu_baseline_sample() if world == 1 and not args.no_cpu else None
    clock_hz = 1e6 * (clk.summary()["sm_mhz"] or 2070.0)
    line = {
        "metric": METRIC, "value": value, "unit": "tests/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (fully determined by n, d, order)",
        "config": {"workload": WORKLOAD_NAME, "codes_per_step": len(probs),
                   "launch": f"{launch_kind}, {ngroups} SM groups",
                   "l2": f"flushed before each step ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "strategies": {f"n={n} d={d} {o}": ("bitmap" if st.strategy == 2 else "distance")
                                  for (n, d, o, w), st in zip(probs, stats_now)}},
        "one_launch_per_code_ms": per_code_ms,
        "one_launch_per_code_ms_per_step": single_ms,
        "batched_speedup_vs_one_launch_per_code": single_ms / mean_step_ms,
        "dense_tests_per_step": dense, "executed_tests_per_step": executed,
        "windows_per_step": sum(st.windows for st in stats_now),
        # the bitmap path's own measure: ball-mark word ORs (L2 atomics) per
        # step and per second of the step; the n = 20 bitmaps are 128 KiB and
        # stay in L2, so no HBM figure applies to them
        "bitmap_marks_per_step": sum(st.marks for st in stats_now),
        "bitmap_marks_per_s": sum(st.marks for st in stats_now) / (mean_step_ms * 1e-3),
        "survivors_per_step": sum(st.survivors for st in stats_now),
        "phase_ms_cta0": {f"n={n} d={d} {o}": dict(
            {ph: (c if ph in ("rounds", "blocks") else round(1e3 * c / clock_hz, 4))
             for ph, c in zip(G.Stats.PHASES, st.phase_cycles)},
            windows=st.windows, survivors=st.survivors, pair_windows=st.pair_windows,
            pair_fallbacks=st.pair_fallbacks)
            for (n, d, o, w), st in zip(probs, stats_now)},
        "e2e": {"value": e2e_value, "unit": "tests/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h,
                "ms_per_step": 1e3 * statistics.mean(e2e_times) if e2e_times else None},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "tests/s",
                     "frac": achieved / peak,
                     "traffic": recorded_traffic() if not args.only else None,
                     "kernel": "gc::sweep_kernel",
                     "peak_source": "gc_probe_test_rate (register-operand XOR+popcount+compare, "
                                    "measured in this run)"},
        "clocks": clk.summary(),
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 300, about 1 s; 5 for --impl reference)")
    ap.add_argument("--warmup", type=int, default=None,
                    help="untimed warm-up steps (default: 10; 3 for --impl reference)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline sample")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-API leg")
    ap.add_argument("--groups", type=int, default=None,
                    help="SM groups of the batched launch (default: one per code)")
    ap.add_argument("--only", default=None,
                    help="run one code instead of the workload, e.g. '24,8,lex' (profiling)")
    args = ap.parse_args()
    ref = args.impl == "reference"
    if args.steps is None:
        args.steps = 5 if ref else 300
    if args.warmup is None:
        args.warmup = 3 if ref else 10
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
