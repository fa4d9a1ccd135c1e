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
    # bm_options: pointer, 4 int32, 3 pointers, 2 int32
    assert ctypes.sizeof(binding.bm_options) == 8 + 16 + 24 + 8
    assert ctypes.sizeof(binding.bm_csr) == 8 + 8 + 8 + 8 + 8 + 8
    assert binding.bm_graph.stats.offset == ctypes.sizeof(binding.bm_graph) - ctypes.sizeof(binding.bm_stats)
    assert ctypes.sizeof(binding.bm_instance) == 32


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
    printf("%zu %zu %zu\n", offsetof(bm_options, want_dists), offsetof(bm_stats, dist_max_rel_err),
           offsetof(bm_csr, dists));
    printf("%zu %zu\n", offsetof(bm_options, centring), offsetof(bm_stats, centred));
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
           binding.bm_options.alloc.offset, binding.bm_stats.ms_prep.offset, binding.bm_graph.edges.offset,
           binding.bm_options.want_dists.offset, binding.bm_stats.dist_max_rel_err.offset,
           binding.bm_csr.dists.offset, binding.bm_options.centring.offset, binding.bm_stats.centred.offset]
    assert got == exp


def test_tile_config_table_on_host():
    """Tile configurations are host-side state: list, query, override, reject, reset."""
    _build.build()
    shapes = binding.tile_shapes()
    assert len(shapes) >= 6 and all(s["d_pad"] == 0 for s in shapes)
    for d in (1, 8, 16, 17, 32, 33, 64, 96, 128, 300, 512):
        c = binding.get_tile_config(d)
        assert c["d_pad"] >= d and c["d_pad"] % c["ck"] == 0 and c["d_pad"] % 16 == 0
        assert {k: c[k] for k in ("ck", "nt", "bbuf", "astg")} in [{k: s[k] for k in ("ck", "nt", "bbuf", "astg")}
                                                                   for s in shapes]
    base = binding.get_tile_config(96)
    try:
        binding.set_tile_config(96, dict(d_pad=96, ck=32, nt=128, bbuf=2, astg=8))
        assert binding.get_tile_config(96)["d_pad"] == 96
        for bad in (dict(d_pad=96, ck=64, nt=256, bbuf=1, astg=5),    # 96 is not a multiple of 64
                    dict(d_pad=64, ck=32, nt=128, bbuf=2, astg=8),    # pads below d
                    dict(d_pad=96, ck=32, nt=256, bbuf=2, astg=8),    # does not fit in shared memory
                    dict(d_pad=96, ck=32, nt=96, bbuf=2, astg=8)):    # not a compiled shape
            with pytest.raises(binding.BallMapperError):
                binding.set_tile_config(96, bad)
        assert binding.get_tile_config(96)["d_pad"] == 96              # a rejected call changes nothing
    finally:
        binding.set_tile_config(96, None)
    assert binding.get_tile_config(96) == base


def test_batch_bounds_rejected_before_the_device():
    """The largest greedy batch is validated with the other arguments, before any device
    call: bm_build takes multiples of 32 up to 16384, bm_build_batched up to 2048."""
    import numpy as np
    _build.build()
    X = np.zeros((4, 2), dtype=np.float32)
    for bad in (16, 33, 16416, 32768):
        with pytest.raises(binding.BallMapperError) as ei:
            binding.bm_build(X, 1.0, batch=bad)
        assert ei.value.status == binding.BM_ERR_ARG
        assert "[32, 16384]" in str(ei.value)
    with pytest.raises(binding.BallMapperError) as ei:
        binding.bm_build_batched([(X, 1.0)], batch=4096)
    assert ei.value.status == binding.BM_ERR_ARG
    assert "[32, 2048]" in str(ei.value)


def test_binding_enums_match_header():
    """The binding's status and path constants equal the header's enum values, and every
    status has a string in the library."""
    text = open(os.path.join(ROOT, "include", "ballmapper.h")).read()
    header = {m.group(1): int(m.group(2))
              for m in re.finditer(r"\b(BM_(?:OK|ERR_\w+|PATH_\w+|CENTRE_\w+))\s*=\s*(\d+)", text)}
    assert len(header) >= 14
    for name, value in header.items():
        assert getattr(binding, name) == value, name
    _build.build()
    lib = binding.load()
    for name, value in header.items():
        if not name.startswith(("BM_PATH", "BM_CENTRE")):
            assert lib.bm_status_string(value), name


def test_centring_mode_rejected_before_the_device():
    """bm_options.centring takes the three bm_centring values; anything else is an
    argument error raised before any device call."""
    import numpy as np
    _build.build()
    lib = binding.load()
    X = np.zeros((4, 2), dtype=np.float32)
    px = X.ctypes.data_as(ctypes.c_void_p)
    for bad in (-1, 3, 7):
        opt = binding._options(lib, "auto", 0, None, True, None)
        opt.centring = bad
        g = binding.bm_graph()
        st = lib.bm_build(px, 4, 2, ctypes.c_float(1.0), ctypes.byref(opt), ctypes.byref(g))
        assert st == binding.BM_ERR_ARG
        assert b"centring" in lib.bm_last_error()
        out, stats = binding.bm_csr(), binding.bm_stats()
        st = lib.bm_range_query(px, 4, 2, px, 4, ctypes.c_float(1.0), ctypes.byref(opt), ctypes.byref(out),
                                ctypes.byref(stats))
        assert st == binding.BM_ERR_ARG
    assert binding.CENTRING == {"auto": 0, "always": 1, "off": 2}


def test_host_result_views_free_once_after_the_last_view():
    """Host results are numpy views of the library's buffers: the buffers go back (one
    free call) only when the last view is gone, and the views read the buffer in place."""
    import gc
    import numpy as np
    calls = []

    def fake_free(obj_ref, opt_ref):
        calls.append(1)

    buf = (ctypes.c_int32 * 8)(*range(8))
    own = binding._HostResult(fake_free, binding.bm_csr(), binding.bm_options())
    a = own.view(ctypes.addressof(buf), ctypes.c_int32, 5)
    b = own.view(ctypes.addressof(buf) + 4 * 5, ctypes.c_int32, 3)
    del own
    gc.collect()
    assert calls == [] and a.tolist() == [0, 1, 2, 3, 4] and b.tolist() == [5, 6, 7]
    buf[1] = 42
    assert a[1] == 42                      # a view, not a copy
    del a
    gc.collect()
    assert calls == []                     # b still holds the buffers
    del b
    gc.collect()
    assert calls == [1]
    empty = binding._HostResult(fake_free, binding.bm_csr(), binding.bm_options()).view(
        ctypes.addressof(buf), ctypes.c_int32, 0)
    assert empty.shape == (0,)
    del empty
    gc.collect()
    assert calls == [1, 1]
