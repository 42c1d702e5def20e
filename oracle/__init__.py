"""CPU oracle for the ordered greedy code sweep -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does; it
shares no code with it.

The arithmetic lives in ``greedy_oracle.c`` (plain C, compiled with gcc into
``oracle/_build/liboracle.so``); this module only compiles it, loads it with
ctypes and marshals numpy arrays.  Each function cites the passage it follows
in the C file's header.

Parity status of each function (the pins are in ``tests/test_oracle.py``):
  order_list / order_sorted  pinned (definitions by comparator, Gray by the
                             reflected construction, brute force)
  greedy_pairwise (O1)       pinned (Example 1 of Section 4.1, Hamming and Golay
                             codes of Section 7, brute force over all subsets)
  greedy_ball (O2)           pinned (equal to O1 wherever O1 runs; Hamming
                             [31,26,3] closed form)
  verify (O3)                pinned (brute force: accepts exactly one subset)
  greedy_selforth            pinned (Section 7: lex gives the extended Golay
                             [24,12,8] and the baby Golay [22,11,6]; the
                             codes are self-dual (Monroe's conjecture, checked
                             where it is claimed); brute force for n <= 4)
  greedy_border              pinned (the standard basis gives lex, the Gray basis
                             gives Gray; B-greedy codes are linear; brute force
                             over all subsets for n <= 4)
  block_test / resolve /     pinned (brute force on small lists; resolve over the
  ball_mark / scan           whole order equals O1; the greedy code's balls
                             cover every candidate; scan of an empty map is the
                             order itself)
  product64                  pinned (the example of Section 5: the self-orthogonal
                             [8,4] code times Code[4,4] is a self-orthogonal
                             [12,5,4] code; brute-force minimum distance of
                             products of small random codes)
  order_list64 / greedy64 /  pinned (equal to the 32-bit forms for n <= 12; the
  verify64 (n <= 64)         disjoint-block closed form of constant-weight codes
                             with d = 2w at n = 33..64 in all four orders; O3
                             accepts the output and rejects perturbations)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

LEX, GRAY, GRLEX, GREVLEX = 0, 1, 2, 3
ORDERS = {"lex": LEX, "gray": GRAY, "grlex": GRLEX, "grevlex": GREVLEX}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "greedy_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: no -march, no intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, u32p, i64p = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p
            lib.orc_candidate_count.restype = ctypes.c_uint64
            lib.orc_candidate_count.argtypes = [i32, i32]
            lib.orc_order_list.restype = i64
            lib.orc_order_list.argtypes = [i32, i32, i32, u32p, i64]
            lib.orc_order_sorted.restype = i64
            lib.orc_order_sorted.argtypes = [i32, i32, i32, u32p, i64]
            for f in (lib.orc_greedy_pairwise, lib.orc_greedy_ball, lib.orc_greedy_selforth):
                f.restype = i64
                f.argtypes = [i32, i32, i32, i32, u32p, i64p, i64]
            lib.orc_greedy_border.restype = i64
            lib.orc_greedy_border.argtypes = [i32, i32, u32p, i32, u32p, i64p, i64]
            lib.orc_border_vector.restype = ctypes.c_uint32
            lib.orc_border_vector.argtypes = [i32, u32p, ctypes.c_uint64]
            lib.orc_verify.restype = i32
            lib.orc_verify.argtypes = [i32, i32, i32, i32, u32p, i64]
            lib.orc_distance.restype = i32
            lib.orc_distance.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            lib.orc_block_test.restype = None
            lib.orc_block_test.argtypes = [i32, u32p, i64, u32p, i64, u32p]
            lib.orc_resolve.restype = i64
            lib.orc_resolve.argtypes = [i32, u32p, i64, i64p]
            lib.orc_ball_mark.restype = i32
            lib.orc_ball_mark.argtypes = [i32, i32, u32p, i64, u32p]
            lib.orc64_candidate_count.restype = ctypes.c_uint64
            lib.orc64_candidate_count.argtypes = [i32, i32]
            lib.orc64_order_list.restype = i64
            lib.orc64_order_list.argtypes = [i32, i32, i32, u32p, i64]
            lib.orc64_greedy.restype = i64
            lib.orc64_greedy.argtypes = [i32, i32, i32, i32, i32, u32p, i64p, i64]
            lib.orc64_verify.restype = i32
            lib.orc64_verify.argtypes = [i32, i32, i32, i32, u32p, i64]
            lib.orc64_product.restype = i64
            lib.orc64_product.argtypes = [u32p, i64, u32p, i64, i32, i32, u32p, i64]
            lib.orc_scan.restype = i64
            lib.orc_scan.argtypes = [i32, i32, i32, u32p, ctypes.c_uint64, ctypes.c_uint64,
                                     u32p, i64]
            _lib = lib
    return _lib


def _ord(ordering) -> int:
    return ORDERS[ordering] if isinstance(ordering, str) else int(ordering)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def candidate_count(n: int, w: int = -1) -> int:
    return int(_load().orc_candidate_count(n, w))


def order_list(n: int, ordering, w: int = -1) -> np.ndarray:
    """Candidates in order, streaming form (Section 4.2)."""
    cnt = candidate_count(n, w)
    out = np.empty(cnt, dtype=np.uint32)
    k = _load().orc_order_list(n, _ord(ordering), w, _ptr(out), cnt)
    if k != cnt:
        raise RuntimeError(f"order_list returned {k}, expected {cnt}")
    return out


def order_sorted(n: int, ordering, w: int = -1) -> np.ndarray:
    """Candidates in order by comparator sort over the whole space (n <= 24)."""
    cnt = candidate_count(n, w)
    out = np.empty(cnt, dtype=np.uint32)
    k = _load().orc_order_sorted(n, _ord(ordering), w, _ptr(out), cnt)
    if k != cnt:
        raise RuntimeError(f"order_sorted returned {k}, expected {cnt}")
    return out


def _greedy(fn, n, d, ordering, w, with_pos):
    lib = _load()
    cap = min(candidate_count(n, w), 1 << 26)
    out = np.empty(max(cap, 1), dtype=np.uint32)
    pos = np.empty(max(cap, 1), dtype=np.int64) if with_pos else None
    k = fn(n, d, _ord(ordering), w, _ptr(out), _ptr(pos) if with_pos else None, cap)
    if k < 0:
        raise RuntimeError(f"oracle error {k} for n={n} d={d} ord={ordering} w={w}")
    if with_pos:
        return out[:k].copy(), pos[:k].copy()
    return out[:k].copy()


def greedy_pairwise(n: int, d: int, ordering="lex", w: int = -1, with_pos: bool = False):
    """O1: each candidate against every codeword so far (Section 4)."""
    return _greedy(_load().orc_greedy_pairwise, n, d, ordering, w, with_pos)


def greedy_ball(n: int, d: int, ordering="lex", w: int = -1, with_pos: bool = False):
    """O2: the same greedy through radius-(d-1) exclusion balls over vectors."""
    return _greedy(_load().orc_greedy_ball, n, d, ordering, w, with_pos)


def greedy_selforth(n: int, d: int, ordering="lex", w: int = -1, with_pos: bool = False):
    """Self-orthogonal greedy (Section 4.4): the pairwise greedy with the
    extra constraint that every codeword is orthogonal to itself and to every
    earlier codeword."""
    return _greedy(_load().orc_greedy_selforth, n, d, ordering, w, with_pos)


def greedy_border(n: int, d: int, basis, w: int = -1, with_pos: bool = False):
    """Greedy over the B-ordering of an ordered basis (Section 4.3): rank r is
    the XOR of basis[j] over the set bits j of r."""
    b = np.ascontiguousarray(np.asarray(basis, dtype=np.uint32))
    if len(b) != n:
        raise ValueError("basis must have n vectors")
    cap = min((1 << n) if w < 0 else candidate_count(n, w), 1 << 26)
    out = np.empty(max(cap, 1), dtype=np.uint32)
    pos = np.empty(max(cap, 1), dtype=np.int64) if with_pos else None
    k = _load().orc_greedy_border(n, d, _ptr(b), w, _ptr(out), _ptr(pos) if with_pos else None,
                                  cap)
    if k < 0:
        raise RuntimeError(f"oracle error {k} (basis dependent or bad arguments)")
    return (out[:k].copy(), pos[:k].copy()) if with_pos else out[:k].copy()


def border_vector(n: int, basis, r: int) -> int:
    b = np.ascontiguousarray(np.asarray(basis, dtype=np.uint32))
    return int(_load().orc_border_vector(n, _ptr(b), r))


def verify(n: int, d: int, ordering, w: int, L) -> int:
    """O3: 0 iff L is exactly the greedy output (see the C header)."""
    L = np.ascontiguousarray(np.asarray(L, dtype=np.uint32))
    return int(_load().orc_verify(n, d, _ord(ordering), w, _ptr(L), len(L)))


def block_test(d: int, cand, code) -> np.ndarray:
    """alive[i] = 1 iff cand[i] is at distance >= d from every codeword."""
    c = np.ascontiguousarray(np.asarray(cand, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(code, dtype=np.uint32))
    alive = np.empty(max(len(c), 1), dtype=np.uint8)
    _load().orc_block_test(d, _ptr(c), len(c), _ptr(k), len(k), _ptr(alive))
    return alive[:len(c)].copy()


def resolve(d: int, cand) -> np.ndarray:
    """List indices the greedy accepts when the list is walked in order."""
    c = np.ascontiguousarray(np.asarray(cand, dtype=np.uint32))
    idx = np.empty(max(len(c), 1), dtype=np.int64)
    k = _load().orc_resolve(d, _ptr(c), len(c), _ptr(idx))
    return idx[:k].copy()


def ball_mark(n: int, d: int, code, bitmap=None) -> np.ndarray:
    """OR the radius-(d-1) balls of the codewords into a 2^n-bit map."""
    k = np.ascontiguousarray(np.asarray(code, dtype=np.uint32))
    if bitmap is None:
        bitmap = np.zeros(max(((1 << n) + 31) // 32, 1), dtype=np.uint32)
    rc = _load().orc_ball_mark(n, d, _ptr(k), len(k), _ptr(bitmap))
    if rc != 0:
        raise RuntimeError(f"oracle ball_mark error {rc}")
    return bitmap


def scan(n: int, ordering, w: int, bitmap, rank0: int, count: int):
    """Vectors of ranks [rank0, rank0+count) whose bit is clear, in order."""
    b = np.ascontiguousarray(np.asarray(bitmap, dtype=np.uint32))
    out = np.empty(max(count, 1), dtype=np.uint32)
    k = _load().orc_scan(n, _ord(ordering), w, _ptr(b), rank0, count, _ptr(out), count)
    if k < 0:
        raise RuntimeError(f"oracle scan error {k}")
    return out[:k].copy()


def dense_tests(positions: np.ndarray, n_candidates: int) -> int:
    """Candidate-codeword distance tests a sweep with no early exit performs:
    the codeword accepted at candidate index p is compared with every later
    candidate, so the total is the sum over codewords of (N - 1 - p)."""
    p = np.asarray(positions, dtype=np.int64)
    return int((n_candidates - 1 - p).sum())


# ---- vectors of up to 64 coordinates (uint64 words) -----------------------
def candidate_count64(n: int, w: int = -1) -> int:
    return int(_load().orc64_candidate_count(n, w))


def order_list64(n: int, ordering, w: int = -1) -> np.ndarray:
    """Candidates in order, by sorting the candidate set with the order's
    comparator (Section 4.2 orders, n <= 64)."""
    cnt = candidate_count64(n, w)
    out = np.empty(max(cnt, 1), dtype=np.uint64)
    k = _load().orc64_order_list(n, _ord(ordering), w, _ptr(out), cnt)
    if k != cnt:
        raise RuntimeError(f"order_list64 returned {k}, expected {cnt}")
    return out[:cnt].copy()


def greedy64(n: int, d: int, ordering="lex", w: int = -1, orth: bool = False,
             with_pos: bool = False):
    """The greedy of Section 4 for n <= 64 (orth: with the Section 4.4
    constraint), pairwise over the sorted candidate list."""
    cap = max(min(candidate_count64(n, w), 1 << 26), 1)
    out = np.empty(cap, dtype=np.uint64)
    pos = np.empty(cap, dtype=np.int64) if with_pos else None
    k = _load().orc64_greedy(n, d, _ord(ordering), w, int(bool(orth)), _ptr(out),
                             _ptr(pos) if with_pos else None, cap)
    if k < 0:
        raise RuntimeError(f"oracle error {k} for n={n} d={d} ord={ordering} w={w}")
    return (out[:k].copy(), pos[:k].copy()) if with_pos else out[:k].copy()


def verify64(n: int, d: int, ordering, w: int, L) -> int:
    """O3 for n <= 64: 0 iff L is exactly the greedy output."""
    L = np.ascontiguousarray(np.asarray(L, dtype=np.uint64))
    return int(_load().orc64_verify(n, d, _ord(ordering), w, _ptr(L), len(L)))


def product64(A, B, len_a: int, len_b: int) -> np.ndarray:
    """Cartesian product of two codes (Section 5, recursion for
    self-orthogonal codes): (a << len_b) | b for every a in A (outer) and b
    in B (inner)."""
    a = np.ascontiguousarray(np.asarray(A, dtype=np.uint64))
    b = np.ascontiguousarray(np.asarray(B, dtype=np.uint64))
    out = np.empty(max(len(a) * len(b), 1), dtype=np.uint64)
    k = _load().orc64_product(_ptr(a), len(a), _ptr(b), len(b), len_a, len_b, _ptr(out),
                              len(out))
    if k < 0:
        raise RuntimeError("product: words do not fit 64 bits")
    return out[:k].copy()
