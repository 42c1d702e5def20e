"""Benchmark of the ordered greedy code sweep on one GB300 (or N replicas).

Workload (one "step"): the nine large codes n=31, d=3 and n=32, d=4 in lex,
Gray, graded-lex and graded-reverse-lex order (2^31 and 2^32 candidates, the
exclusion-bitmap path with 256 / 512 MiB of bits) and n=28, d=5 lex, each
one whole sweep over its candidates, one launch per code on the whole GPU,
in the strategy the planner picks.  Metric: candidate-codeword distance tests
per second, counted as dense-equivalent tests (for each candidate, the number
of codewords accepted before it -- the tests a sweep without early exit
performs, the paper's naive kernel) divided by the device time; the wall time
per code is reported beside it, as the paper reports it (Section 6, Table 1).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs the same
workload as an independent replica (the sweep of one code does not shard).
Besides the headline, the line carries: the same codes through the C ABI's
synchronous call into pinned host buffers (e2e), the five-code workload
n=24 d=8 lex + n=20 d=4 in four orders as one batched launch, the 512
seeded instances as one batch against one launch each, a short served
replay, and CPU baselines (the oracle single-threaded on a bounded sample,
and per instance on every host core over the 512 instances).
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

WORKLOAD = [(31, 3, "lex"), (31, 3, "gray"), (31, 3, "grlex"), (31, 3, "grevlex"),
            (32, 4, "lex"), (32, 4, "gray"), (32, 4, "grlex"), (32, 4, "grevlex"),
            (28, 5, "lex")]
WORKLOAD_NAME = ("n=31 d=3 and n=32 d=4 in lex, gray, grlex and grevlex order + n=28 d=5 lex "
                 "(9 whole sweeps, one launch each)")
SMALL = [(24, 8, "lex"), (20, 4, "lex"), (20, 4, "gray"), (20, 4, "grlex"), (20, 4, "grevlex")]
SMALL_NAME = "n=24 d=8 lex + n=20 d=4 x {lex, gray, grlex, grevlex}"
METRIC = "candidate-codeword distance tests/s (dense-equivalent)"
# bounded CPU sample of the workload: its one code the single-thread oracle
# finishes in seconds (the n = 31 and 32 codes take minutes to an hour each)
CPU_SAMPLE = (28, 5, "lex")
L2_FLUSH_BYTES = 256 << 20
HBM_FALLBACK_GBS = 6800.0


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


def name(code) -> str:
    n, d, o = code[:3]
    return f"n={n} d={d} {o}"


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
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU legs
def oracle_sample():
    """The single-thread exclusion-ball oracle on the workload's bounded
    sample: (dense tests, seconds)."""
    import oracle
    oracle.build()
    n, d, o = CPU_SAMPLE
    t = time.perf_counter()
    _, pos = oracle.greedy_ball(n, d, o, with_pos=True)
    dt = time.perf_counter() - t
    return oracle.dense_tests(pos, 1 << n), dt


def _one_instance(p):
    import oracle
    n, d, o, w = p
    t = time.perf_counter()
    code = oracle.greedy_ball(n, d, o, w)
    return len(code), time.perf_counter() - t


def cpu_parallel_baseline():
    """The 512 seeded batch instances, each through the exclusion-ball oracle,
    spread over every host core (a spawned process pool)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    import oracle
    from paper_1507_05398_gb300.workloads import batch_instances
    oracle.build()
    probs = batch_instances()
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    with ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_one_instance, probs, chunksize=1))
    wall = time.perf_counter() - t
    return {"value": len(probs) / wall, "unit": "codes/s", "cores": cores, "kind": "oracle",
            "sample": f"the {len(probs)} seeded batch instances (exclusion-ball oracle, one "
                      f"process per core, {wall:.1f} s wall, "
                      f"{sum(r[1] for r in res):.1f} s of CPU)",
            "cpu": cpu_model()}


# ------------------------------------------------------------------ reference
def run_reference(args):
    """The CPU oracle, single-threaded, as it stands, on the bounded sample of
    the workload (one step = one whole n=28 d=5 lex sweep)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    dense = 0
    seconds = 0.0
    for i in range(args.warmup + args.steps):
        dn, dt = oracle_sample()
        if i >= args.warmup:
            dense += dn
            seconds += dt
    value = dense / seconds
    sample = (f"{name(CPU_SAMPLE)}, exclusion-ball oracle, whole sweep per step "
              f"({seconds / args.steps:.1f} s)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "tests/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * seconds / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (fully determined by n, d, order)",
        "config": {"workload": WORKLOAD_NAME, "parallelism": "host, 1 thread",
                   "sample": name(CPU_SAMPLE)},
        "cpu_baseline": {"value": value, "unit": "tests/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "tests/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours
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


def kernel_source_hash(files=None) -> str:
    """Hash of CUDA/C++ sources' code (comments and layout ignored): recorded
    DRAM traffic stays valid across comment-only edits.  Default: every
    source of the library."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_1507_05398_gb300", "csrc")
    if files is None:
        files = sorted(glob.glob(os.path.join(csrc, "*.cu")) +
                       glob.glob(os.path.join(csrc, "*.cuh")) +
                       glob.glob(os.path.join(csrc, "*.h")))
    else:
        files = [os.path.join(csrc, f) for f in files]
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        h.update(_code_only(open(f, encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


GRID_SOURCES = ["gc_gridsweep.cu", "gc_block.cuh", "gc_device.cuh"]
SWEEP_SOURCES = ["gc_sweep.cu", "gc_block.cuh", "gc_device.cuh"]   # sweep_kernel (captures)


def recorded_traffic(profile: str, files=None):
    """DRAM bytes per launch from a committed ncu summary, or None if the
    kernel's sources changed since that capture."""
    p = os.path.join(ROOT, "profiles", profile)
    try:
        txt = open(p).read()
    except OSError:
        return None
    vals = dict(l.split(":", 1) for l in txt.splitlines()
                if l.startswith(("traffic_bytes_per_launch:", "kernel_source_sha256_16:")))
    if vals.get("kernel_source_sha256_16", "").strip() != kernel_source_hash(files):
        return None
    return int(vals["traffic_bytes_per_launch"].strip())


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of the GB300s if
    the measurement file is present, else the stated fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d:
                v = d[k]
                v = v.get("value", v) if isinstance(v, dict) else v
                return float(v), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, TypeError):
        pass
    return HBM_FALLBACK_GBS, "fallback (no MEASURED_PEAKS.json in this run)"


def algorithmic_bytes(n: int, codewords: int) -> int:
    """The bitmap path's algorithmic bytes for one code: the 2^n-bit map
    written once (zero fill) and read once (the lookups), every one of its
    32-byte sectors marked at least once, and 4 bytes per codeword out."""
    bitmap = (1 << n) // 8
    return 3 * bitmap + 4 * codewords


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
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # resident buffers: output, statistics and workspace of every code
    bufs = []
    for n, d, o in WORKLOAD:
        cap = G.capacity_bound(n, d, -1)
        ws_bytes = G.workspace_size(n, d, o, -1)
        ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
        base = (-ws.data_ptr()) % 256
        bufs.append((n, d, o, torch.empty(cap, dtype=torch.int32, device=dev),
                     torch.zeros(ctypes.sizeof(G.Stats), dtype=torch.uint8, device=dev),
                     ws[base:base + ws_bytes]))

    def one_step(events=None):
        for k, (n, d, o, out, st, ws) in enumerate(bufs):
            if events is not None:
                events[k][0].record(stream)
            G.generate_async(n, d, o, -1, out=out, stats=st, workspace=ws, stream=stream)
            if events is not None:
                events[k][1].record(stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        one_step()
    torch.cuda.synchronize()
    stats = [G.stats_from(st) for *_, st, _ws in bufs]
    for s, c in zip(stats, WORKLOAD):
        if s.status != 0:
            raise RuntimeError(f"sweep failed for {name(c)}: {s.as_dict()}")
    dense = sum(s.dense_tests for s in stats)
    executed = sum(s.executed_tests for s in stats)
    marks = sum(s.marks for s in stats)
    launches_per_step = 2 * len(WORKLOAD)  # the ball table and the sweep, per code

    # timed region: K steps, L2 flushed before each, CUDA events per code
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in WORKLOAD] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.fill_(s & 0xff)
            one_step(ev[s])
        torch.cuda.synchronize()
    code_ms = [[a.elapsed_time(b) for a, b in step] for step in ev]
    step_ms = [sum(x) for x in code_ms]
    mean_step_ms = statistics.mean(step_ms)
    if world > 1:
        t = torch.tensor([mean_step_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        mean_step_ms = float(t.item())
    value = world * dense / (mean_step_ms * 1e-3)
    per_code_ms = {name(c): statistics.mean(x[k] for x in code_ms)
                   for k, c in enumerate(WORKLOAD)}
    stats = [G.stats_from(st) for *_, st, _ws in bufs]
    strategies = {1: "distance", 2: "bitmap", 3: "grid bitmap"}
    clock_hz = 1e6 * (clk.summary()["sm_mhz"] or 2070.0)

    # end to end through the C ABI's synchronous call: gc_generate into a
    # pinned host buffer (its scratch allocation, the sweep, the copy of the
    # code back to the host and the frees are all inside the timed call)
    e2e_times, d2h = [], 0
    e2e_steps = 0 if args.no_e2e else min(args.steps, 3)
    if e2e_steps:
        # pinned host buffers of each code's size (known from the runs above)
        hosts = [torch.empty(max(s.codewords, 1), dtype=torch.int32, pin_memory=True)
                 for s in stats]
        L = G.lib()
        for s in range(1 + e2e_steps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            got = []
            for (n, d, o), h in zip(WORKLOAD, hosts):
                cnt = ctypes.c_uint64(h.numel())
                rc = L.gc_generate(n, d, G.ORDERS[o], -1, ctypes.c_void_p(h.data_ptr()),
                                   ctypes.byref(cnt))
                if rc != 0:
                    raise G.GcError(rc, "gc_generate")
                got.append(int(cnt.value))
            if s >= 1:
                e2e_times.append(time.perf_counter() - t)
        if got != [st.codewords for st in stats]:
            raise RuntimeError("end-to-end code sizes differ from the device-resident run")
        d2h = sum(4 * c + ctypes.sizeof(G.Stats) for c in got)
        del hosts
    e2e_value = world * dense / statistics.mean(e2e_times) if e2e_times else None

    # the bitmap roofline: algorithmic bytes per step over the event time
    peak_gbs, peak_src = hbm_peak()
    alg = sum(algorithmic_bytes(n, s.codewords) for (n, d, o), s in zip(WORKLOAD, stats))
    achieved_gbs = alg / (mean_step_ms * 1e-3) / 1e9
    mark_peak = G.probe_mark_rate()
    test_peak, _ = G.probe_test_rate()
    marks_per_s = marks / (mean_step_ms * 1e-3)
    chain_us = {name(c): 1e3 * per_code_ms[name(c)] / max(s.windows, 1)
                for c, s in zip(WORKLOAD, stats)}
    # DRAM bytes per grid-sweep launch, averaged over the nine codes (one
    # 1-pass ncu capture of the whole step); only for the full workload
    traffic_launch = (None if args.only else
                      recorded_traffic("grid_sweep_bench_workload_dram.md", GRID_SOURCES))

    extra = {}
    if not args.only and not args.no_extras:
        extra = extras(args, G, torch, stream, flush, test_peak)
    del bufs
    torch.cuda.empty_cache()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu:
        dn, dt = oracle_sample()
        cpu = {"value": dn / dt, "unit": "tests/s", "cores": 1, "kind": "oracle",
               "sample": f"{name(CPU_SAMPLE)} (exclusion-ball oracle, one whole sweep, {dt:.1f} s)",
               "cpu": cpu_model()}
    line = {
        "metric": METRIC, "value": value, "unit": "tests/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (fully determined by n, d, order)",
        "config": {"workload": WORKLOAD_NAME, "codes_per_step": len(WORKLOAD),
                   "launch": "one cooperative launch per code on the whole GPU (gc_generate_async)",
                   "l2": f"inputs larger than L2 (256 / 512 MiB bitmaps) and flushed before each "
                         f"step ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "strategies": {name(c): strategies.get(s.strategy, str(s.strategy))
                                  for c, s in zip(WORKLOAD, stats)}},
        "wall_ms_per_code": per_code_ms,
        "codewords_per_code": {name(c): s.codewords for c, s in zip(WORKLOAD, stats)},
        "dense_tests_per_step": dense, "executed_tests_per_step": executed,
        "executed_tests_per_s": executed / (mean_step_ms * 1e-3),
        "bitmap_marks_per_step": marks, "bitmap_marks_per_s": marks_per_s,
        "windows_per_code": {name(c): s.windows for c, s in zip(WORKLOAD, stats)},
        "survivors_per_code": {name(c): s.survivors for c, s in zip(WORKLOAD, stats)},
        "e2e": {"value": e2e_value, "unit": "tests/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h,
                "ms_per_step": 1e3 * statistics.mean(e2e_times) if e2e_times else None,
                "steps": len(e2e_times),
                "call": "gc_generate(n, d, ordering, -1, pinned host buffer, &count) per code: "
                        "scratch allocation, sweep, copy of the code to the host, frees; "
                        "inputs are four integers per code (no host-to-device copy)"},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
                     "frac": achieved_gbs / peak_gbs,
                     "traffic": None if traffic_launch is None else traffic_launch,
                     "kernel": "gc::grid_sweep_kernel",
                     "peak_source": peak_src,
                     "algorithmic_bytes_per_step": alg},
        "roofline_by_strategy": {
            "bitmap_hbm": {"achieved_gbs": achieved_gbs, "peak_gbs": peak_gbs,
                           "frac": achieved_gbs / peak_gbs},
            "bitmap_marks": {"achieved_ors_per_s": marks_per_s, "peak_ors_per_s": mark_peak,
                             "frac": marks_per_s / mark_peak,
                             "peak_source": "gc_probe_mark_rate (random word ORs in a 64 MiB "
                                            "region, measured in this run)"},
            "bitmap_window_chain_us": chain_us,
            "distance": extra.get("distance_roofline"),
        },
        "clocks": clk.summary(),
    }
    for k, v in extra.items():
        if k != "distance_roofline":
            line[k] = v
    if cpu is not None:
        line["cpu_baseline"] = cpu
        if not args.no_extras and not args.only:
            line["cpu_parallel_baseline"] = cpu_parallel_baseline()
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def extras(args, G, torch, stream, flush, test_peak):
    """The smaller workloads: the five-code batch (and its distance job alone
    for the distance roofline), the 512 seeded instances batched against one
    launch each, and a short served replay."""
    out = {}
    reps = max(3, min(args.steps, 20))
    # five codes in one batched launch, replayed from a CUDA graph
    probs = [(n, d, o, -1) for n, d, o in SMALL]
    batch = G.BatchBuffers(probs, ngroups=len(probs))
    batch.launch(stream)
    torch.cuda.synchronize()
    graph = batch.capture()
    for _ in range(3):
        graph.replay()
    ts = []
    for s in range(reps):
        flush.fill_(s & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.replay()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    res = batch.results()
    small_ms = statistics.mean(ts)
    one = {}
    for (n, d, o, w) in probs:
        cap = G.capacity_bound(n, d, w)
        outb = torch.empty(cap, dtype=torch.int32, device=flush.device)
        st = torch.zeros(ctypes.sizeof(G.Stats), dtype=torch.uint8, device=flush.device)
        wsz = G.workspace_size(n, d, o, w)
        ws = torch.empty(wsz + 256, dtype=torch.uint8, device=flush.device)
        base = (-ws.data_ptr()) % 256
        wsa = ws[base:base + wsz]
        G.generate_async(n, d, o, w, out=outb, stats=st, workspace=wsa, stream=stream)
        tt = []
        for s in range(reps):
            flush.fill_(s & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            G.generate_async(n, d, o, w, out=outb, stats=st, workspace=wsa, stream=stream)
            b.record(stream)
            b.synchronize()
            tt.append(a.elapsed_time(b))
        one[f"n={n} d={d} {o}"] = statistics.mean(tt)
        if (n, d, o) == (24, 8, "lex"):
            s = G.stats_from(st)
            rate = s.executed_tests / (one[f"n={n} d={d} {o}"] * 1e-3)
            out["distance_roofline"] = {
                "code": "n=24 d=8 lex, alone on the whole GPU",
                "achieved_tests_per_s": rate, "peak_tests_per_s": test_peak,
                "frac": rate / test_peak,
                "peak_source": "gc_probe_test_rate (register-operand XOR+popcount+compare, "
                               "measured in this run)"}
    out["workload_n24d8_n20d4"] = {
        "workload": SMALL_NAME + " as one batched persistent launch (CUDA graph replay)",
        "ms_per_step": small_ms,
        "dense_tests_per_s": sum(st.dense_tests for _, st in res) / (small_ms * 1e-3),
        "one_launch_per_code_ms": one,
        "batched_speedup_vs_one_launch_per_code": sum(one.values()) / small_ms}
    del batch, graph

    # the 512 seeded instances: one batch against one launch each
    from paper_1507_05398_gb300.workloads import batch_instances
    inst = batch_instances()
    b512 = G.BatchBuffers(inst)
    b512.launch(stream)
    torch.cuda.synchronize()
    g512 = b512.capture()
    g512.replay()
    torch.cuda.synchronize()
    tb = []
    for s in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g512.replay()
        b.record(stream)
        b.synchronize()
        tb.append(a.elapsed_time(b))
    r512 = b512.results()
    bad = [p for (c, st), p in zip(r512, inst) if st.status != 0]
    if bad:
        raise RuntimeError(f"batch instances failed: {bad[:3]}")
    batch_ms = statistics.mean(tb)
    # one launch each, on preallocated buffers (workspace of the largest)
    caps = [G.capacity_bound(n, d, w) for n, d, o, w in inst]
    outb = torch.empty(max(caps), dtype=torch.int32, device=flush.device)
    st = torch.zeros(ctypes.sizeof(G.Stats), dtype=torch.uint8, device=flush.device)
    wsz = max(G.workspace_size(n, d, o, w) for n, d, o, w in inst)
    ws = torch.empty(wsz + 256, dtype=torch.uint8, device=flush.device)
    base = (-ws.data_ptr()) % 256
    wsa = ws[base:base + wsz]
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for (n, d, o, w), cap in zip(inst, caps):
        G.generate_async(n, d, o, w, out=outb[:cap], stats=st, workspace=wsa, stream=stream)
    b.record(stream)
    b.synchronize()
    single_ms = a.elapsed_time(b)
    out["batch512_ms"] = batch_ms
    out["batch512_one_launch_each_ms"] = single_ms
    out["batch512_vs_one_launch"] = single_ms / batch_ms
    out["batch512_codes_per_s"] = len(inst) / (batch_ms * 1e-3)
    out["batch512_workload"] = ("512 seeded instances (numpy PCG64 seed 1507): n~U{14..24}, "
                                "d~U{3..8}, four orders, 25% constant weight w~U{3..n/2}; one "
                                "persistent launch (CUDA graph replay) vs one launch per code")
    del b512, g512, ws, outb
    torch.cuda.synchronize()

    # a short served replay (continuous batching)
    from paper_1507_05398_gb300.serve import capacity, replay
    from paper_1507_05398_gb300.workloads import serve_requests
    nreq, load, seed = args.serve_requests, 0.8, 1507
    with G.Server(max_n=28, pool_bytes=8 << 30, queue_capacity=2048) as srv:
        probe = [p for _, p in serve_requests(512, seed + 1, 1.0)]
        cap_jobs = capacity(srv, probe)
        rate = load * cap_jobs
        stream_req = serve_requests(nreq, seed, rate)
        lat, makespan = replay(srv, stream_req)
    lat_ms = sorted(1e3 * x for x in lat)
    q = lambda f: lat_ms[min(len(lat_ms) - 1, int(f * len(lat_ms)))]  # noqa: E731
    out["serve_p50_ms"] = q(0.50)
    out["serve_p99_ms"] = q(0.99)
    out["serve_jobs_per_s"] = nreq / makespan
    out["serve_capacity_jobs_per_s"] = cap_jobs
    out["serve_workload"] = (f"{nreq} seeded Poisson requests (seed {seed}) at {load} x the "
                             f"measured capacity (lambda = {rate:.0f} jobs/s): 95% like the batch "
                             "instances, 5% n~U{26..28} d~U{3,4}")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 3; 3 for --impl reference)")
    ap.add_argument("--warmup", type=int, default=None,
                    help="untimed warm-up steps (default: 3)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baselines")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-API leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the smaller workloads (batch, 512 instances, serving)")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the served replay (default 2000)")
    ap.add_argument("--only", default=None,
                    help="run one code instead of the workload, e.g. '31,3,lex' (profiling)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 3
    if args.warmup is None:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
