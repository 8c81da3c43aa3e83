"""The C-ABI library loads and exports every entry point include/gp.h declares,
and its host-side argument checks work without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "gp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(gp_[a-z_0-9]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_16012_gb300 import _build

    _build.build()
    import paper_2010_16012_gb300 as gp

    return gp.load()


def test_every_declared_symbol_exported(lib):
    import paper_2010_16012_gb300 as gp

    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in gp.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_static_text_and_defaults(lib):
    import paper_2010_16012_gb300 as gp

    assert lib.gp_version() == 1
    for st in range(0, -7, -1):
        assert lib.gp_status_string(st)
    o = gp.default_options()
    assert o.pull_light_max > 0 and o.chunk_edges >= 32 and o.bfs_alpha > 0


def test_struct_sizes_match_header():
    import paper_2010_16012_gb300 as gp

    # layouts fixed by include/gp.h (x86-64 and AArch64 agree)
    assert ctypes.sizeof(gp.gp_options) == 64
    assert ctypes.sizeof(gp.gp_pr_stats) == 56
    assert ctypes.sizeof(gp.gp_kernel_time) == 64
    assert ctypes.sizeof(gp.gp_graph_info) == 88
    assert ctypes.sizeof(gp.gp_bfs_summary) == 32


def test_struct_layouts_match_c_compiler(tmp_path):
    """Sizes and field offsets of the binding's ctypes structures equal those the
    C compiler derives from include/gp.h."""
    import shutil
    import subprocess

    import paper_2010_16012_gb300 as gp

    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"gp_options": gp.gp_options, "gp_pr_stats": gp.gp_pr_stats, "gp_bfs_stats": gp.gp_bfs_stats, "gp_bfs_summary": gp.gp_bfs_summary,
               "gp_batch_stats": gp.gp_batch_stats, "gp_tune_result": gp.gp_tune_result, "gp_sssp_stats": gp.gp_sssp_stats, "gp_tc_stats": gp.gp_tc_stats, "gp_fe_stats": gp.gp_fe_stats, "gp_bc_stats": gp.gp_bc_stats,
               "gp_kernel_time": gp.gp_kernel_time, "gp_graph_info": gp.gp_graph_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gp.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        name, field, val = line.split()
        cls = structs[name]
        want = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert int(val) == want, (name, field, int(val), want)
        seen += 1
    assert seen > 30


def test_host_argument_checks(lib):
    import paper_2010_16012_gb300 as gp

    h = ctypes.c_void_p()
    st = lib.gp_graph_upload(ctypes.byref(h), -1, 0, None, None, None, None, None, None, 0, None)
    assert st == gp.ERR_INVALID and not h.value
    assert b"outside" in lib.gp_last_error()
    st = lib.gp_graph_upload(ctypes.byref(h), 4, 0, None, None, None, None, None, None, 0, None)
    assert st == gp.ERR_INVALID
    st = lib.gp_pagerank(None, 0, 0.85, 10, 0.0, None, None, None, None, None)
    assert st == gp.ERR_INVALID
    st = lib.gp_bfs(None, 0, 0, None, None, None, None)
    assert st == gp.ERR_INVALID
    st = lib.gp_bfs_multi(None, None, 1, 0, None, None, 0, None, None)
    assert st == gp.ERR_INVALID
    assert lib.gp_graph_free(None) == gp.OK
    assert lib.gp_options_default(None) == gp.ERR_INVALID


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: a missing libgp.so raises instead of degrading."""
    import paper_2010_16012_gb300 as gp

    saved = gp._lib
    gp._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            gp.load(str(tmp_path / "nope.so"))
    finally:
        gp._lib = saved
