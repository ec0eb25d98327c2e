"""The C-ABI library loads on a machine without a GPU and exports every function that
include/cc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(cc_[a-z_0-9]+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    d = _declared()
    for n in ["cc_context_create", "cc_context_destroy", "cc_graph_load", "cc_graph_free", "cc_enumerate",
              "cc_batch_submit", "cc_batch_poll", "cc_status_str", "cc_get_limits"]:
        assert n in d


def test_library_exports_every_declared_symbol():
    from paper_1410_4876_gb300 import build, cc
    build.build()
    lib = ctypes.CDLL(cc.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    for n in cc.SIGNATURES:
        assert n in _declared(), n


def test_status_strings_and_limits():
    from paper_1410_4876_gb300 import cc
    cc.load_library()
    assert cc.status_str(cc.CC_ERR_INVALID_GRAPH) == "not a simple undirected graph"
    lim = cc.cc_get_limits()
    assert lim.max_n_bitset == 256 and lim.max_n_batch == 64 and lim.max_n_csr >= 2000


def test_struct_layouts_match_header(tmp_path):
    # the ctypes mirrors of the option, result and tuner structs have the C layout
    import shutil
    import subprocess

    from paper_1410_4876_gb300 import cc
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"cc_options": cc.cc_options, "cc_run_info": cc.cc_run_info, "cc_tune_result": cc.cc_tune_result,
               "cc_cycles": cc.cc_cycles, "cc_serve_options": cc.cc_serve_options,
               "cc_completion": cc.cc_completion}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cc.h"', "int main(void) {"]
    for name, py in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        name, field, value = line.split()
        py = structs[name]
        got = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert got == int(value), (name, field, got, value)


def test_null_handles_are_refused_without_a_gpu():
    # argument checks run before any CUDA call: NULL handles, outputs and sinks give
    # CC_ERR_ARG on a machine without a GPU
    from paper_1410_4876_gb300 import cc
    lib = cc.load_library()
    u64 = ctypes.c_uint64(0)
    hist = (ctypes.c_uint64 * 8)()
    assert lib.cc_enumerate(None, 0, hist, ctypes.byref(u64), None, None, None) == cc.CC_ERR_ARG
    assert lib.cc_enumerate_stream(None, 0, 1 << 20, 1 << 24, None, None, hist, ctypes.byref(u64), None, None,
                                   None) == cc.CC_ERR_ARG
    sink = cc.CYCLE_SINK(lambda *a: None)
    assert lib.cc_enumerate_stream(None, 0, 1 << 20, 1 << 24, ctypes.cast(sink, ctypes.c_void_p), None, hist,
                                   ctypes.byref(u64), None, None, None) == cc.CC_ERR_ARG
    handle = ctypes.c_void_p()
    rp = (ctypes.c_uint32 * 2)(0, 0)
    assert lib.cc_graph_load(None, 1, rp, rp, ctypes.byref(handle)) == cc.CC_ERR_ARG
    assert lib.cc_context_set_options(None, ctypes.byref(cc.cc_options())) == cc.CC_ERR_ARG
    assert lib.cc_tune(None, 0, None, ctypes.byref(cc.cc_tune_result())) == cc.CC_ERR_ARG
    assert lib.cc_get_trace(None, 0, None, None, ctypes.byref(u64)) == cc.CC_ERR_ARG
    lib.cc_graph_free(None)
    lib.cc_context_destroy(None)
