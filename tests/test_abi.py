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
