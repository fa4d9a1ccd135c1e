"""The C-ABI library builds, loads without a GPU and exports every symbol the
public header declares (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2601_01405_gb300 import _build, binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names += re.findall(r"BM_API\s+[\w\s\*]+?\b(bm_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("bm_build", "bm_range_query", "bm_graph_free", "bm_csr_free", "bm_last_error"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_loads_and_reports_version():
    _build.build()
    assert binding.version() >= 100
    lib = binding.load()
    assert lib.bm_status_string(binding.BM_ERR_ARG) == b"invalid argument"


def test_struct_layouts_match_header():
    # bm_options: pointer, 4 int32, 3 pointers
    assert ctypes.sizeof(binding.bm_options) == 8 + 16 + 24
    assert ctypes.sizeof(binding.bm_csr) == 8 + 8 + 8 + 8 + 8
    assert binding.bm_graph.stats.offset == ctypes.sizeof(binding.bm_graph) - ctypes.sizeof(binding.bm_stats)


def test_struct_layouts_match_c_compiler(tmp_path):
    """sizeof/offsetof of the public structs as gcc sees them equal the binding's ctypes layout."""
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "ballmapper.h"
int main(void) {
    printf("%zu %zu %zu %zu %zu\n", sizeof(bm_options), sizeof(bm_stats), sizeof(bm_csr), sizeof(bm_graph),
           offsetof(bm_graph, stats));
    printf("%zu %zu %zu\n", offsetof(bm_options, alloc), offsetof(bm_stats, ms_prep), offsetof(bm_graph, edges));
    return 0;
}
''')
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)]).decode().split()
    got = [int(v) for v in out]
    exp = [ctypes.sizeof(binding.bm_options), ctypes.sizeof(binding.bm_stats), ctypes.sizeof(binding.bm_csr),
           ctypes.sizeof(binding.bm_graph), binding.bm_graph.stats.offset,
           binding.bm_options.alloc.offset, binding.bm_stats.ms_prep.offset, binding.bm_graph.edges.offset]
    assert got == exp
