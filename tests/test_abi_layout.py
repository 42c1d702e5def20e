"""The binding's ctypes structures match include/gc.h field for field: the
header is compiled with the host C compiler, which reports every struct's
size and every field's offset, and those must equal ctypes' (no GPU)."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1507_05398_gb300 as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PAIRS = [(G.Problem, "gc_problem"), (G.Plan, "gc_plan_t"), (G.Stats, "gc_stats"),
         (G.Job, "gc_job"), (G.ServerConfig, "gc_server_config")]


def _c_layout(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gc.h"', "int main(void) {"]
    for cls, cname in PAIRS:
        lines.append(f'    printf("{cname} %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{cname}.{field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return dict(line.rsplit(" ", 1) for line in out.splitlines())


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a host C compiler")
def test_struct_sizes_and_offsets_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for cls, cname in PAIRS:
        assert int(c[cname]) == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert int(c[f"{cname}.{field}"]) == getattr(cls, field).offset, (cname, field)
