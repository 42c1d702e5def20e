"""ctypes binding of libgc (include/gc.h): argument marshalling only.

Every step of the sweep runs in the CUDA kernels of libgc.so; nothing here
computes codes.  Device buffers are torch CUDA tensors; the stream is torch's
current stream unless one is given.  If the library is missing the import of
any entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

__all__ = [
    "LEX", "GRAY", "GRLEX", "GREVLEX", "BASIS", "NO_WEIGHT", "ORDERS",
    "CONSTRAINT_NONE", "CONSTRAINT_SELF_ORTHOGONAL",
    "STRATEGY_AUTO", "STRATEGY_DISTANCE", "STRATEGY_BITMAP", "STRATEGY_BITMAP_GRID",
    "GcError", "Problem", "Plan", "Stats", "lib", "library_path", "header_functions",
    "strerror", "candidate_count", "capacity_bound", "plan", "workspace_size",
    "generate", "generate_async", "generate_host",
    "workspace_size64", "generate64", "generate64_async", "generate64_host",
    "product", "selforth_product",
    "unrank", "rank", "block_test", "resolve", "bitmap_mark", "bitmap_scan",
    "probe_test_rate", "probe_mark_rate", "stats_from", "generate_noalloc", "noalloc_scratch_bytes",
    "Job", "BatchBuffers", "batch_workspace_size", "batch_generate_async", "generate_batch",
    "batch_result_bytes", "clear_batch_cache",
    "ServerConfig", "Server", "autotune", "batch_autotune", "set_tune_cache",
]

LEX, GRAY, GRLEX, GREVLEX, BASIS = 0, 1, 2, 3, 4
NO_WEIGHT = -1
ORDERS = {"lex": LEX, "gray": GRAY, "grlex": GRLEX, "grevlex": GREVLEX, "basis": BASIS}
STRATEGY_AUTO, STRATEGY_DISTANCE, STRATEGY_BITMAP, STRATEGY_BITMAP_GRID = 0, 1, 2, 3
_STRAT = {None: 0, "auto": 0, "distance": 1, "bitmap": 2, "grid": 3}

_HERE = os.path.dirname(os.path.abspath(__file__))
_HEADER = os.path.join(os.path.dirname(_HERE), "include", "gc.h")


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libgc.so")


class GcError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code}): {_last_error()}")


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("d", ctypes.c_int), ("ordering", ctypes.c_int),
                ("weight", ctypes.c_int), ("constraint", ctypes.c_int),
                ("basis", ctypes.POINTER(ctypes.c_uint32))]


CONSTRAINT_NONE, CONSTRAINT_SELF_ORTHOGONAL = 0, 1
_CONSTRAINTS = {None: 0, "none": 0, "self_orthogonal": 1, "selforth": 1}


def _constraint(c):
    return _CONSTRAINTS[c] if (c is None or isinstance(c, str)) else int(c)


class Plan(ctypes.Structure):
    _fields_ = [("strategy", ctypes.c_int), ("grid", ctypes.c_int), ("block", ctypes.c_int),
                ("window_min", ctypes.c_uint32), ("window_max", ctypes.c_uint32),
                ("survivor_target", ctypes.c_uint32)]


class Job(ctypes.Structure):
    _fields_ = [("prob", Problem), ("strategy", ctypes.c_int), ("d_out", ctypes.c_void_p),
                ("capacity", ctypes.c_uint64), ("d_stats", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("codewords", ctypes.c_uint64), ("candidates", ctypes.c_uint64),
                ("dense_tests", ctypes.c_uint64), ("executed_tests", ctypes.c_uint64),
                ("marks", ctypes.c_uint64), ("windows", ctypes.c_uint64),
                ("survivors", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("strategy", ctypes.c_int32), ("phase_cycles", ctypes.c_uint64 * 12),
                ("pair_windows", ctypes.c_uint64), ("pair_fallbacks", ctypes.c_uint64)]

    PHASES = ("mark", "generate", "test_new", "test_old", "wait", "gather", "resolve", "commit",
              "res_matrix", "res_rounds", "res_append_kill", "rounds")

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "phase_cycles"}
        d["phase_cycles"] = dict(zip(self.PHASES, list(self.phase_cycles)))
        return d


_lock = threading.Lock()
_lib = None

_u64, _i32, _u32, _vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p
_SIGS = {
    "gc_strerror": (ctypes.c_char_p, [_i32]),
    "gc_last_error": (ctypes.c_char_p, []),
    "gc_candidate_count": (_u64, [_i32, _i32, _i32]),
    "gc_capacity_bound": (_u64, [_i32, _i32, _i32]),
    "gc_plan": (_i32, [ctypes.POINTER(Problem), ctypes.POINTER(Plan)]),
    "gc_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(Problem), ctypes.POINTER(Plan)]),
    "gc_generate": (_i32, [_i32, _i32, _i32, _i32, _vp, ctypes.POINTER(_u64)]),
    "gc_generate_async": (_i32, [ctypes.POINTER(Problem), ctypes.POINTER(Plan), _vp, _u64, _vp,
                                 _vp, ctypes.c_size_t, _vp]),
    "gc_unrank": (_i32, [_i32, _i32, _i32, _u64, _u64, _vp, _vp]),
    "gc_rank": (_i32, [_i32, _i32, _vp, _u64, _vp, _vp]),
    "gc_block_test": (_i32, [_i32, _vp, _u64, _vp, _u64, _vp, _vp]),
    "gc_resolve": (_i32, [_i32, _vp, _u32, _vp, _vp, _vp]),
    "gc_bitmap_mark": (_i32, [_i32, _i32, _vp, _u64, _vp, _vp]),
    "gc_bitmap_scan": (_i32, [_i32, _i32, _i32, _vp, _u64, _u64, _vp, _u64, _vp, _vp]),
    "gc_probe_test_rate": (_i32, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "gc_probe_mark_rate": (_i32, [ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]),
    "gc_generate_noalloc": (_i32, [ctypes.POINTER(Problem), ctypes.POINTER(Plan), _vp, _u64, _vp,
                                   _vp]),
    "gc_batch_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(Job), _i32, _i32]),
    "gc_server_create": (_i32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "gc_server_submit": (_i32, [_vp, ctypes.POINTER(Problem), _i32, ctypes.POINTER(_u64)]),
    "gc_server_poll": (_i32, [_vp, ctypes.POINTER(_u64), _i32, ctypes.POINTER(_i32)]),
    "gc_server_fetch": (_i32, [_vp, _u64, _vp, ctypes.POINTER(_u64), ctypes.c_void_p]),
    "gc_server_release": (_i32, [_vp, _u64]),
    "gc_server_destroy": (_i32, [_vp]),
    "gc_autotune": (_i32, [ctypes.POINTER(Problem), ctypes.POINTER(Plan),
                           ctypes.POINTER(ctypes.c_double)]),
    "gc_set_tune_cache": (_i32, [ctypes.c_char_p]),
    "gc_batch_autotune": (_i32, [ctypes.POINTER(Job), _i32, _i32, _i32, ctypes.POINTER(_i32)]),
    "gc_batch_generate_async": (_i32, [ctypes.POINTER(Job), _i32, _i32, _vp, ctypes.c_size_t, _vp]),
    "gc_batch_create": (_i32, [ctypes.POINTER(Job), _i32, _i32, _vp, ctypes.c_size_t, _vp,
                               ctypes.POINTER(ctypes.c_void_p)]),
    "gc_batch_launch": (_i32, [_vp, _vp]),
    "gc_batch_destroy": (_i32, [_vp]),
    "gc_noalloc_scratch_bytes": (ctypes.c_size_t, []),
    "gc_workspace_size64": (ctypes.c_size_t, [ctypes.POINTER(Problem), ctypes.POINTER(Plan)]),
    "gc_product": (_i32, [_vp, _u64, _i32, _vp, _u64, _i32, _vp, _u64, _vp]),
    "gc_product64": (_i32, [_vp, _u64, _i32, _vp, _u64, _i32, _vp, _u64, _vp]),
    "gc_generate64": (_i32, [_i32, _i32, _i32, _i32, _vp, ctypes.POINTER(_u64)]),
    "gc_generate64_async": (_i32, [ctypes.POINTER(Problem), ctypes.POINTER(Plan), _vp, _u64, _vp,
                                   _vp, ctypes.c_size_t, _vp]),
}


def header_functions() -> list[str]:
    """Names of the functions include/gc.h declares."""
    text = open(_HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gc_[a-z_0-9]+)\s*\(", text)))


def lib():
    """Load libgc.so (build it first if a toolchain is present)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                from . import build as _build
                _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().gc_strerror(code).decode()


def _last_error() -> str:
    return lib().gc_last_error().decode()


def _check(rc: int, what: str):
    if rc != 0:
        raise GcError(rc, what)


def _ord(o) -> int:
    if isinstance(o, (list, tuple, np.ndarray)):
        return BASIS
    return ORDERS[o] if isinstance(o, str) else int(o)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _dev_u32(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype in (torch.int32, torch.uint32)):
        raise TypeError("expected a CUDA tensor of 32-bit words")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t


# ---------------------------------------------------------------- information
def candidate_count(n: int, weight: int = NO_WEIGHT, ordering="lex") -> int:
    return int(lib().gc_candidate_count(n, weight, _ord(ordering)))


def capacity_bound(n: int, d: int, weight: int = NO_WEIGHT) -> int:
    return int(lib().gc_capacity_bound(n, d, weight))


def _bound(n, d, weight, constraint):
    b = capacity_bound(n, d, weight)
    if _constraint(constraint) == CONSTRAINT_SELF_ORTHOGONAL:
        b = min(b, 1 << (n // 2))
    return b


def _problem(n, d, ordering, weight, constraint=None):
    """ordering: a name, an ordering code, or -- for a B-ordering (Section
    4.3) -- the list of n basis vectors b_1..b_n."""
    p = Problem(n, d, _ord(ordering), weight, _constraint(constraint), None)
    if p.ordering == BASIS:
        arr = (ctypes.c_uint32 * n)(*[int(v) for v in ordering])
        p.basis = ctypes.cast(arr, ctypes.POINTER(ctypes.c_uint32))
        p._basis_keepalive = arr
    return p


def plan(n: int, d: int, ordering="lex", weight: int = NO_WEIGHT, constraint=None) -> Plan:
    p = Plan()
    _check(lib().gc_plan(ctypes.byref(_problem(n, d, ordering, weight, constraint)),
                         ctypes.byref(p)), "gc_plan")
    return p


def _plan_arg(strategy=None, **kw):
    if strategy is None and not kw:
        return None
    p = Plan()
    p.strategy = _STRAT.get(strategy, strategy or 0)
    for k, v in kw.items():
        if v is not None:
            setattr(p, k, v)
    return p


def workspace_size(n, d, ordering="lex", weight=NO_WEIGHT, strategy=None, constraint=None,
                   **plan_kw) -> int:
    pl = _plan_arg(strategy, **plan_kw)
    return int(lib().gc_workspace_size(ctypes.byref(_problem(n, d, ordering, weight, constraint)),
                                       ctypes.byref(pl) if pl is not None else None))


# ---------------------------------------------------------------- the sweep
def generate_async(n, d, ordering="lex", weight=NO_WEIGHT, *, out, stats, workspace,
                   strategy=None, stream=None, constraint=None, **plan_kw):
    """gc_generate_async: out (uint32 CUDA tensor, its length is the capacity),
    stats (uint8 CUDA tensor of sizeof(gc_stats) bytes), workspace (uint8 CUDA
    tensor of >= workspace_size bytes, 256-byte aligned)."""
    pl = _plan_arg(strategy, **plan_kw)
    rc = lib().gc_generate_async(ctypes.byref(_problem(n, d, ordering, weight, constraint)),
                                 ctypes.byref(pl) if pl is not None else None,
                                 _ptr(out), out.numel() if out is not None else 0, _ptr(stats),
                                 _ptr(workspace), workspace.numel(), _stream(stream))
    _check(rc, "gc_generate_async")


def generate_noalloc(n, d, ordering="lex", weight=NO_WEIGHT, *, out, stats, strategy=None,
                     stream=None, constraint=None, **plan_kw):
    """gc_generate_noalloc: like generate_async but the library allocates
    nothing -- its scratch is a static device array (see include/gc.h).  For
    callers that cannot allocate device memory when they need a code."""
    pl = _plan_arg(strategy, **plan_kw)
    rc = lib().gc_generate_noalloc(ctypes.byref(_problem(n, d, ordering, weight, constraint)),
                                   ctypes.byref(pl) if pl is not None else None,
                                   _ptr(out), out.numel() if out is not None else 0, _ptr(stats),
                                   _stream(stream))
    _check(rc, "gc_generate_noalloc")


def noalloc_scratch_bytes() -> int:
    return int(lib().gc_noalloc_scratch_bytes())




def _flat_layout(njobs, caps):
    """Byte offsets of each output in a batch's flat buffer (statistics
    first, 256-byte aligned pieces) and the buffer's size."""
    al = lambda v: (v + 255) & ~255  # noqa: E731
    offs, off = [], al(njobs * ctypes.sizeof(Stats))
    for c in caps:
        offs.append(off)
        off += al(4 * max(c, 1))
    return offs, off


def batch_result_bytes(problems) -> int:
    """Bytes one results() call copies back for this batch."""
    ps = [tuple(p) + (None,) * (6 - len(p)) for p in problems]
    return _flat_layout(len(ps), [_bound(n, d, w, c) for n, d, o, w, _, c in ps])[1]


class BatchBuffers:
    """Device buffers (outputs, stats, workspace) for a batch of problems,
    prepared once (gc_batch_create) and launched any number of times
    (gc_batch_launch), directly or as a captured CUDA graph.

    problems: list of (n, d, ordering, weight[, strategy[, constraint]]).
    The statistics and every output live in one device buffer (so results()
    is one copy back, into a pinned host buffer); allocated once through
    torch's caching allocator."""

    def __init__(self, problems, ngroups=0, device=None):
        import torch
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.problems = [tuple(p) + (None,) * (6 - len(p)) for p in problems]
        self.ngroups = ngroups
        self.caps = [_bound(n, d, w, c) for n, d, o, w, _, c in self.problems]
        nj, sbytes = len(self.problems), ctypes.sizeof(Stats)
        self._offs, off = _flat_layout(nj, self.caps)
        self._flat = torch.zeros(off, dtype=torch.uint8, device=dev)
        self._host = torch.empty(off, dtype=torch.uint8, pin_memory=True)
        self.stats = self._flat[:nj * sbytes].view(nj, sbytes)
        self.outs = [self._flat[o:o + 4 * max(c, 1)].view(torch.int32)
                     for o, c in zip(self._offs, self.caps)]
        self.jobs = (Job * len(self.problems))()
        for k, (n, d, o, w, st, c) in enumerate(self.problems):
            j = self.jobs[k]
            j.prob = _problem(n, d, o, w, c)
            j.strategy = _STRAT.get(st, st or 0)
            j.d_out = self.outs[k].data_ptr()
            j.capacity = self.caps[k]
            j.d_stats = self.stats[k].data_ptr()
        ws_bytes = batch_workspace_size(self.jobs, ngroups)
        if ws_bytes == 0:
            raise GcError(1, "gc_batch_workspace_size")
        ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
        base = (-ws.data_ptr()) % 256
        self._ws_alloc = ws
        self.workspace = ws[base:base + ws_bytes]
        self._handle = ctypes.c_void_p()
        _check(lib().gc_batch_create(self.jobs, len(self.jobs), ngroups, _ptr(self.workspace),
                                     self.workspace.numel(), _stream(None),
                                     ctypes.byref(self._handle)), "gc_batch_create")
        # launches may come on any stream: the workspace is filled first
        torch.cuda.current_stream().synchronize()

    def launch(self, stream=None):
        """gc_batch_launch: one run of the whole batch (one kernel launch)."""
        _check(lib().gc_batch_launch(self._handle, _stream(stream)), "gc_batch_launch")

    def capture(self):
        """A torch.cuda.CUDAGraph holding one launch of the batch; replay()
        reruns it with no host work."""
        import torch
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.launch()
        return g

    def __del__(self):
        h = getattr(self, "_handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.gc_batch_destroy(h)
            self._handle = None

    def results(self, stream=None):
        """[(code uint32 numpy array, Stats)]: one copy of the statistics and
        the outputs back to the host, ordered after the work on `stream`
        (default: the current stream), which it then waits for."""
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            self._host.copy_(self._flat, non_blocking=True)
        st.synchronize()
        h = self._host.numpy()
        sbytes = ctypes.sizeof(Stats)
        out = []
        for k in range(len(self.problems)):
            s = Stats.from_buffer_copy(h[k * sbytes:(k + 1) * sbytes].tobytes())
            m = min(s.codewords, self.caps[k])
            code = h[self._offs[k]:self._offs[k] + 4 * m].view(np.uint32).copy()
            out.append((code, s))
        return out


def batch_workspace_size(jobs, ngroups=0) -> int:
    return int(lib().gc_batch_workspace_size(jobs, len(jobs), ngroups))


def batch_generate_async(jobs, ngroups, workspace, stream=None):
    _check(lib().gc_batch_generate_async(jobs, len(jobs), ngroups, _ptr(workspace),
                                         workspace.numel(), _stream(stream)),
           "gc_batch_generate_async")


_batch_cache: dict = {}
_batch_lock = threading.Lock()
_BATCH_CACHE_SIZE = 4


def clear_batch_cache():
    """Drops the prepared batches generate_batch keeps (and their memory)."""
    with _batch_lock:
        _batch_cache.clear()


def generate_batch(problems, ngroups=0, stream=None):
    """Generate many codes in one launch; returns [(code, Stats)] with the
    codes as host arrays.  The prepared batch (plan, workspace, ball tables,
    buffers) is kept for the next call with the same problems, grouping,
    device and GC_* environment (the last few such sets; clear_batch_cache()
    drops them), so a repeated call is one launch and one copy back."""
    import torch
    key = (tuple(tuple(p) for p in problems), ngroups, torch.cuda.current_device(),
           tuple(sorted((k, v) for k, v in os.environ.items() if k.startswith("GC_"))))
    with _batch_lock:
        buf = _batch_cache.pop(key, None)
        if buf is None:
            buf = BatchBuffers(problems, ngroups)
        _batch_cache[key] = buf  # most recent last
        while len(_batch_cache) > _BATCH_CACHE_SIZE:
            _batch_cache.pop(next(iter(_batch_cache)))
        buf.launch(stream)
        return buf.results(stream)


def stats_from(t) -> Stats:
    """Decode a stats tensor (device or host) into a Stats struct."""
    raw = bytes(t.cpu().numpy().tobytes())
    return Stats.from_buffer_copy(raw[:ctypes.sizeof(Stats)])


def generate(n, d, ordering="lex", weight=NO_WEIGHT, *, strategy=None, stream=None,
             capacity=None, return_stats=False, constraint=None, **plan_kw):
    """Whole sweep on the current CUDA device; returns a CUDA tensor with the
    code in acceptance order (and the Stats if asked): int32 words for
    n <= 32, int64 words (the uint64 bit patterns, generate64) for n > 32."""
    if n > 32:
        return generate64(n, d, ordering, weight, strategy=strategy, stream=stream,
                          capacity=capacity, return_stats=return_stats, constraint=constraint,
                          **plan_kw)
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    cap = _bound(n, d, weight, constraint) if capacity is None else capacity
    ws_bytes = workspace_size(n, d, ordering, weight, strategy, constraint, **plan_kw)
    if ws_bytes == 0:
        raise GcError(1, "gc_workspace_size")
    out = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    st = torch.zeros(ctypes.sizeof(Stats), dtype=torch.uint8, device=dev)
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
    base = (-ws.data_ptr()) % 256
    ws_al = ws[base:base + ws_bytes]
    generate_async(n, d, ordering, weight, out=out[:cap] if cap else None, stats=st,
                   workspace=ws_al, strategy=strategy, stream=stream, constraint=constraint,
                   **plan_kw)
    s = stats_from(st)
    if s.status != 0:
        raise GcError(int(s.status), "sweep")
    code = out[:min(s.codewords, cap)]
    return (code, s) if return_stats else code


def generate_host(n, d, ordering="lex", weight=NO_WEIGHT, capacity=None) -> np.ndarray:
    """gc_generate with a host buffer (the library allocates and copies)."""
    cap = capacity_bound(n, d, weight) if capacity is None else capacity
    buf = np.empty(max(cap, 1), dtype=np.uint32)
    cnt = _u64(cap)
    rc = lib().gc_generate(n, d, _ord(ordering), weight,
                           buf.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt))
    _check(rc, "gc_generate")
    return buf[:cnt.value].copy()


# ---------------------------------------------------------------- wide vectors
def workspace_size64(n, d, ordering="lex", weight=NO_WEIGHT, strategy=None, constraint=None,
                     **plan_kw) -> int:
    pl = _plan_arg(strategy, **plan_kw)
    return int(lib().gc_workspace_size64(
        ctypes.byref(_problem(n, d, ordering, weight, constraint)),
        ctypes.byref(pl) if pl is not None else None))


def generate64_async(n, d, ordering="lex", weight=NO_WEIGHT, *, out, stats, workspace,
                     strategy=None, stream=None, constraint=None, **plan_kw):
    """gc_generate64_async (n <= 64): out is an int64 CUDA tensor (uint64 bit
    patterns; its length is the capacity), stats and workspace as for
    generate_async (workspace_size64 bytes)."""
    import torch
    if out is not None and out.dtype not in (torch.int64, torch.uint64):
        raise TypeError("expected a CUDA tensor of 64-bit words")
    pl = _plan_arg(strategy, **plan_kw)
    rc = lib().gc_generate64_async(ctypes.byref(_problem(n, d, ordering, weight, constraint)),
                                   ctypes.byref(pl) if pl is not None else None,
                                   _ptr(out), out.numel() if out is not None else 0, _ptr(stats),
                                   _ptr(workspace), workspace.numel(), _stream(stream))
    _check(rc, "gc_generate64_async")


def generate64(n, d, ordering="lex", weight=NO_WEIGHT, *, strategy=None, stream=None,
               capacity=None, return_stats=False, constraint=None, **plan_kw):
    """Whole wide sweep (n <= 64); returns an int64 CUDA tensor holding the
    uint64 codewords in acceptance order (and the Stats if asked)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    cap = _bound(n, d, weight, constraint) if capacity is None else capacity
    ws_bytes = workspace_size64(n, d, ordering, weight, strategy, constraint, **plan_kw)
    if ws_bytes == 0:
        raise GcError(1, "gc_workspace_size64")
    out = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
    st = torch.zeros(ctypes.sizeof(Stats), dtype=torch.uint8, device=dev)
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
    base = (-ws.data_ptr()) % 256
    generate64_async(n, d, ordering, weight, out=out[:cap] if cap else None, stats=st,
                     workspace=ws[base:base + ws_bytes], strategy=strategy, stream=stream,
                     constraint=constraint, **plan_kw)
    s = stats_from(st)
    if s.status != 0:
        raise GcError(int(s.status), "sweep")
    code = out[:min(s.codewords, cap)]
    return (code, s) if return_stats else code


def generate64_host(n, d, ordering="lex", weight=NO_WEIGHT, capacity=None) -> np.ndarray:
    """gc_generate64 with a host buffer; returns uint64 words."""
    cap = capacity_bound(n, d, weight) if capacity is None else capacity
    buf = np.empty(max(cap, 1), dtype=np.uint64)
    cnt = _u64(cap)
    rc = lib().gc_generate64(n, d, _ord(ordering), weight,
                             buf.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt))
    _check(rc, "gc_generate64")
    return buf[:cnt.value].copy()


# ---------------------------------------------------------------- products
def product(a, len_a: int, b, len_b: int, out=None, stream=None):
    """gc_product / gc_product64 (Section 5, recursion for self-orthogonal
    codes): every codeword of a (length len_a) followed by every codeword of b
    (length len_b), a outermost.  a and b are CUDA tensors of one word width
    (int32: len_a + len_b <= 32, int64: <= 64); returns a tensor of that
    width with len(a) * len(b) words."""
    import torch
    if a.dtype != b.dtype or a.element_size() not in (4, 8) or not (a.is_cuda and b.is_cuda):
        raise TypeError("expected two CUDA tensors of the same 32- or 64-bit word type")
    a, b = a.contiguous(), b.contiguous()
    total = a.numel() * b.numel()
    if out is None:
        out = torch.empty(max(total, 1), dtype=a.dtype, device=a.device)
    f = lib().gc_product64 if a.element_size() == 8 else lib().gc_product
    _check(f(_ptr(a), a.numel(), len_a, _ptr(b), b.numel(), len_b, _ptr(out), out.numel(),
             _stream(stream)), "gc_product")
    return out[:total]


def selforth_product(n: int, d: int, k: int, stream=None):
    """Code[n, d] built as Section 5 does: the lex self-orthogonal greedy code
    of length n - k times the one of length k (both from the sweep, then one
    gc_product).  Word width as generate() gives for length n."""
    if not (1 <= k < n):
        raise ValueError("need 1 <= k < n")
    gen = generate64 if n > 32 else generate
    a = gen(n - k, d, "lex", constraint="self_orthogonal", stream=stream)
    b = gen(k, d, "lex", constraint="self_orthogonal", stream=stream)
    return product(a, n - k, b, k, stream=stream)


# ---------------------------------------------------------------- the steps
def unrank(n, ordering, weight, rank0, count, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty(max(count, 1), dtype=torch.int32, device="cuda")
    _check(lib().gc_unrank(n, _ord(ordering), weight, rank0, count, _ptr(_dev_u32(out)),
                           _stream(stream)), "gc_unrank")
    return out[:count]


def rank(n, ordering, vectors, stream=None):
    import torch
    v = _dev_u32(vectors)
    out = torch.empty(max(v.numel(), 1), dtype=torch.int64, device=v.device)
    _check(lib().gc_rank(n, _ord(ordering), _ptr(v), v.numel(), _ptr(out), _stream(stream)),
           "gc_rank")
    return out[:v.numel()]


def block_test(d, cand, code, stream=None):
    import torch
    c = _dev_u32(cand)
    k = _dev_u32(code)
    alive = torch.empty(max(c.numel(), 1), dtype=torch.uint8, device=c.device)
    _check(lib().gc_block_test(d, _ptr(c), c.numel(), _ptr(k), k.numel(), _ptr(alive),
                               _stream(stream)), "gc_block_test")
    return alive[:c.numel()]


def resolve(d, cand, stream=None):
    import torch
    c = _dev_u32(cand)
    acc = torch.empty(max(c.numel(), 1), dtype=torch.int32, device=c.device)
    cnt = torch.zeros(1, dtype=torch.int32, device=c.device)
    _check(lib().gc_resolve(d, _ptr(c), c.numel(), _ptr(acc), _ptr(cnt), _stream(stream)),
           "gc_resolve")
    return acc[:int(cnt.item())]


def bitmap_mark(n, d, code, bitmap=None, stream=None):
    import torch
    k = _dev_u32(code)
    if bitmap is None:
        bitmap = torch.zeros(max(((1 << n) + 31) // 32, 1), dtype=torch.int32, device=k.device)
    _check(lib().gc_bitmap_mark(n, d, _ptr(k), k.numel(), _ptr(_dev_u32(bitmap)),
                                _stream(stream)), "gc_bitmap_mark")
    return bitmap


def bitmap_scan(n, ordering, weight, bitmap, rank0, count, capacity=None, stream=None):
    import torch
    b = _dev_u32(bitmap)
    cap = count if capacity is None else capacity
    out = torch.empty(max(cap, 1), dtype=torch.int32, device=b.device)
    found = torch.zeros(1, dtype=torch.int64, device=b.device)
    _check(lib().gc_bitmap_scan(n, _ord(ordering), weight, _ptr(b), rank0, count, _ptr(out), cap,
                                _ptr(found), _stream(stream)), "gc_bitmap_scan")
    f = int(found.item())
    return out[:min(f, cap)], f


def probe_mark_rate(region_bytes: int = 0) -> float:
    """Bitmap word ORs per second at random words of a region (default 64 MiB)."""
    r = ctypes.c_double(0)
    _check(lib().gc_probe_mark_rate(ctypes.byref(r), region_bytes), "gc_probe_mark_rate")
    return r.value


def probe_test_rate() -> tuple[float, float]:
    """(distance tests per second with register operands, reported SM clock Hz)."""
    r, c = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().gc_probe_test_rate(ctypes.byref(r), ctypes.byref(c)), "gc_probe_test_rate")
    return r.value, c.value


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_n", ctypes.c_int), ("ngroups", ctypes.c_int), ("pool_bytes", ctypes.c_size_t),
                ("queue_capacity", ctypes.c_int), ("store_words", ctypes.c_uint64),
                ("idle_seconds", ctypes.c_double)]


class Server:
    """Continuous-batching request server (gc_server_*): requests are admitted
    by output footprint while others run in the same persistent launch."""

    def __init__(self, max_n=28, ngroups=0, pool_bytes=0, queue_capacity=0, store_words=0,
                 idle_seconds=0.0):
        cfg = ServerConfig(max_n, ngroups, pool_bytes, queue_capacity, store_words, idle_seconds)
        h = ctypes.c_void_p()
        _check(lib().gc_server_create(ctypes.byref(cfg), ctypes.byref(h)), "gc_server_create")
        self._h = h
        self._ids = (_u64 * 4096)()

    def submit(self, n, d, ordering="lex", weight=NO_WEIGHT, strategy=None, constraint=None):
        """Request id, or None if not admitted now (pool or ring full)."""
        rid = _u64(0)
        rc = lib().gc_server_submit(self._h, ctypes.byref(_problem(n, d, ordering, weight,
                                                                   constraint)),
                                    _STRAT.get(strategy, strategy or 0), ctypes.byref(rid))
        if rc == 2:
            return None
        _check(rc, "gc_server_submit")
        return int(rid.value)

    def poll(self):
        nd = _i32(0)
        _check(lib().gc_server_poll(self._h, self._ids, len(self._ids), ctypes.byref(nd)),
               "gc_server_poll")
        return [int(self._ids[k]) for k in range(nd.value)]

    def fetch(self, rid, capacity=None):
        """(code as uint32 numpy array, Stats) of a finished request."""
        st = Stats()
        cnt = _u64(0)
        rc = lib().gc_server_fetch(self._h, rid, None, ctypes.byref(cnt), ctypes.byref(st))
        if rc not in (0, 2):
            _check(rc, "gc_server_fetch")
        buf = np.empty(max(int(cnt.value), 1), dtype=np.uint32)
        cnt2 = _u64(len(buf))
        _check(lib().gc_server_fetch(self._h, rid, buf.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(cnt2), ctypes.byref(st)), "gc_server_fetch")
        return buf[:cnt2.value], st

    def release(self, rid):
        _check(lib().gc_server_release(self._h, rid), "gc_server_release")

    def close(self):
        if self._h:
            _check(lib().gc_server_destroy(self._h), "gc_server_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def autotune(n, d, ordering="lex", weight=NO_WEIGHT, constraint=None):
    """(fastest Plan measured on this device, its time in ms)."""
    best, ms = Plan(), ctypes.c_double(0)
    _check(lib().gc_autotune(ctypes.byref(_problem(n, d, ordering, weight, constraint)),
                             ctypes.byref(best), ctypes.byref(ms)), "gc_autotune")
    return best, ms.value


def batch_autotune(problems, ngroups=0, max_jobs=-1) -> int:
    """gc_batch_autotune: measured plans for the costliest distinct problems
    of a batch, on the CTAs the batch gives each, into the installed tuning
    cache.  problems: (n, d, ordering, weight[, strategy[, constraint]]).
    Returns how many problems were tuned."""
    ps = [tuple(p) + (None,) * (6 - len(p)) for p in problems]
    jobs = (Job * len(ps))()
    for k, (n, d, o, w, st, c) in enumerate(ps):
        jobs[k].prob = _problem(n, d, o, w, c)
        jobs[k].strategy = _STRAT.get(st, st or 0)
    tuned = _i32(0)
    _check(lib().gc_batch_autotune(jobs, len(ps), ngroups, max_jobs, ctypes.byref(tuned)),
           "gc_batch_autotune")
    return int(tuned.value)


def set_tune_cache(path):
    """Install (or with None remove) the plain-text tuning cache."""
    _check(lib().gc_set_tune_cache(path.encode() if path else None), "gc_set_tune_cache")
