"""Host-side helpers of bench.py (no GPU): the source hash that keeps a
recorded ncu traffic figure tied to the kernel it was measured on, the
parsing of that record, the HBM peak's source, and the algorithmic bytes the
bitmap roofline divides by."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_drops_comments_and_layout_but_keeps_literals():
    a = 'int x = 1; // one\n/* block\n comment */ int  y =\n 2; const char* s = "// not a comment";'
    b = 'int x = 1;\nint y = 2;   const char* s = "// not a comment";  // tail'
    assert bench._code_only(a) == bench._code_only(b)
    assert '"// not a comment"' in bench._code_only(a)
    assert bench._code_only("int x = 1;") != bench._code_only("int x = 2;")
    # an escaped quote inside a literal does not end it
    assert bench._code_only(r'char c = "\"//x"; int z;') == r'char c = "\"//x"; int z;'


def test_kernel_source_hash_is_stable_and_covers_the_named_files():
    h1 = bench.kernel_source_hash(bench.GRID_SOURCES)
    h2 = bench.kernel_source_hash(bench.GRID_SOURCES)
    assert h1 == h2 and len(h1) == 16
    assert h1 != bench.kernel_source_hash(bench.SWEEP_SOURCES)
    assert h1 != bench.kernel_source_hash()


def test_recorded_traffic_needs_a_matching_hash(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash(bench.GRID_SOURCES)
    (prof / "ok.md").write_text(f"text\ntraffic_bytes_per_launch: 12345\nkernel_source_sha256_16: {h}\n")
    (prof / "stale.md").write_text("traffic_bytes_per_launch: 12345\nkernel_source_sha256_16: 0000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # kernel_source_hash reads the sources under ROOT: point it back at the repository's
    real = bench.kernel_source_hash
    monkeypatch.setattr(bench, "kernel_source_hash", lambda files=None: h if files == bench.GRID_SOURCES else real(files))
    assert bench.recorded_traffic("ok.md", bench.GRID_SOURCES) == 12345
    assert bench.recorded_traffic("stale.md", bench.GRID_SOURCES) is None
    assert bench.recorded_traffic("missing.md", bench.GRID_SOURCES) is None


def test_hbm_peak_prefers_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    v, src = bench.hbm_peak()
    assert v == bench.HBM_FALLBACK_GBS and src.startswith("fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6779.0}))
    v, src = bench.hbm_peak()
    assert v == 6779.0 and src.startswith("measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("{not json")
    v, src = bench.hbm_peak()
    assert v == bench.HBM_FALLBACK_GBS


def test_algorithmic_bytes_of_the_bench_codes():
    # n = 31: 2^31-bit map filled, read and marked once (3 x 256 MiB), 2^26
    # codewords of 4 bytes out: 1 GiB
    assert bench.algorithmic_bytes(31, 1 << 26) == 3 * (1 << 28) + 4 * (1 << 26) == 1 << 30
    assert bench.algorithmic_bytes(32, 1 << 26) == 3 * (1 << 29) + (1 << 28)
