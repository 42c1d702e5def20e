"""Host-side checks of the C ABI: the library loads, exports every function
include/gc.h declares, and its argument checks and bounds answer without a
GPU (no compute call is made here)."""
import ctypes
from math import comb

import pytest

import paper_1507_05398_gb300 as G


def test_library_exports_every_declared_symbol():
    L = G.lib()
    names = G.header_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    # every declared function also has a binding signature
    from paper_1507_05398_gb300.gc import _SIGS
    assert set(names) == set(_SIGS)


def test_strerror_names_every_code():
    for code in range(0, 8):
        assert G.strerror(code) and G.strerror(code) != "unknown error"
    assert G.strerror(99) == "unknown error"


@pytest.mark.parametrize("n,w,ordname,want", [
    (10, -1, "lex", 1024), (32, -1, "gray", 1 << 32), (12, 5, "lex", comb(12, 5)),
    (12, 5, "grevlex", comb(12, 5)), (12, 5, "gray", comb(12, 5)), (0, -1, "lex", 0),
    (33, -1, "lex", 1 << 33), (40, 3, "gray", comb(40, 3)), (40, -1, "gray", 1 << 40), (35, 7, "grevlex", comb(35, 7)),
    (64, 32, "grlex", comb(64, 32)), (64, -1, "lex", 0), (64, 3, "gray", comb(64, 3)), (12, 5, "basis", 4096), (65, 2, "lex", 0),
    (5, 6, "lex", 0), (5, -2, "lex", 0), (5, -1, 5, 0), (5, -1, 4, 32), (6, 3, 4, 64)])
def test_candidate_count(n, w, ordname, want):
    assert G.candidate_count(n, w, ordname) == want


@pytest.mark.parametrize("n,d,w,want", [
    (15, 3, -1, 2048), (7, 3, -1, 16), (23, 7, -1, 4096), (24, 8, -1, (1 << 24) // 2325),
    (10, 1, -1, 1024), (10, 0, -1, 1024), (10, 2, -1, 1024), (12, 4, 3, comb(12, 3)),
    (32, 4, -1, (1 << 32) // 33), (5, -1, -1, 0), (40, 3, -1, (1 << 40) // 41),
    (64, 4, 2, comb(64, 2)), (35, 8, 7, (1 << 35) // (1 + 35 + comb(35, 2) + comb(35, 3))),
    (64, 3, -1, 0)])
def test_capacity_bound(n, d, w, want):
    assert G.capacity_bound(n, d, w) == want


def test_argument_errors_without_gpu():
    L = G.lib()
    cnt = ctypes.c_uint64(0)
    assert L.gc_generate(0, 3, 0, -1, None, ctypes.byref(cnt)) == 1
    assert L.gc_generate(8, -1, 0, -1, None, ctypes.byref(cnt)) == 1
    assert L.gc_generate(8, 3, 7, -1, None, ctypes.byref(cnt)) == 1
    assert L.gc_generate(8, 3, 0, 9, None, ctypes.byref(cnt)) == 1
    assert "n must be" in G.gc._last_error() or G.gc._last_error()
    p = G.Problem(8, 3, 0, -1)
    assert L.gc_unrank(8, 0, -1, 250, 10, None, None) == 1   # past the rank space
    assert L.gc_resolve(-1, None, 0, None, None, None) == 1
    assert L.gc_plan(None, None) == 1
    assert L.gc_generate_async(ctypes.byref(p), None, None, 0, None, None, 0, None) == 1
    # wide vectors: n > 32 only through the gc_*64 entries
    assert L.gc_generate(33, 3, 0, 2, None, ctypes.byref(cnt)) == 1
    assert "64" in G.gc._last_error()
    assert L.gc_generate64(65, 3, 0, 2, None, ctypes.byref(cnt)) == 1
    assert L.gc_generate64(64, 3, 0, -1, None, ctypes.byref(cnt)) == 1   # 2^64 ranks
    assert L.gc_generate64(64, 3, 1, -1, None, ctypes.byref(cnt)) == 1   # Gray, 2^64 ranks
    assert L.gc_generate64(40, 3, 4, -1, None, ctypes.byref(cnt)) == 1   # no wide B-ordering
    w = G.Problem(40, 3, 0, 4)
    assert L.gc_generate64_async(ctypes.byref(w), None, None, 0, None, None, 0, None) == 1


def test_batch_handle_argument_errors_without_gpu():
    L = G.lib()
    h = ctypes.c_void_p()
    assert L.gc_batch_create(None, 0, 0, None, 0, None, ctypes.byref(h)) == 1   # no jobs
    assert not h.value
    jobs = (G.Job * 1)()
    assert L.gc_batch_create(jobs, 1, 0, None, 0, None, None) == 1              # no handle slot
    assert L.gc_batch_launch(None, None) == 1
    assert L.gc_batch_destroy(None) == 0
    assert L.gc_product(None, 2, 20, None, 2, 13, None, 4, None) == 1            # 33 bits > 32
    assert L.gc_product64(None, 0, 40, None, 0, 24, None, 0, None) == 0          # empty product
    assert L.gc_product64(None, 0, 0, None, 0, 4, None, 0, None) == 1            # len_a = 0
