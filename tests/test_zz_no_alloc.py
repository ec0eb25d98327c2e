"""cc_enumerate_noalloc: the allocation-free entry point, for callers that may not allocate
memory while they run (a plugin or real-time loop whose host application forbids device
allocations after start-up, a process whose device memory belongs to another pool
allocator, a latency-critical path that cannot afford an allocation's device-wide
synchronisation).  It must give exactly what cc_enumerate gives, call after call, although
every call reuses the same fixed device array.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1410_4876_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1410_4876_gb300 import cc as _cc
    _cc.load_library()
    return _cc


def _noalloc(cc, g, max_len=0):
    lib = cc.load_library()
    L = g.n if (max_len == 0 or max_len > g.n) else max_len
    hist = np.zeros(L + 1, dtype=np.uint64)
    tc = np.zeros(L + 1, dtype=np.uint64)
    h = ctypes.c_uint64(0)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint32)
    cl = np.ascontiguousarray(g.col if g.col.size else np.zeros(1, np.uint32), dtype=np.uint32)
    s = lib.cc_enumerate_noalloc(g.n, cc._p32(rp), cc._p32(cl), max_len, None, cc._p64(hist), ctypes.byref(h),
                                 cc._p64(tc))
    return s, hist, int(h.value), tc


@pytest.mark.parametrize("g,max_len", [(I.grid(6, 6), 0), (I.gnp(60, 0.15, 7), 0), (I.grid(8, 8), 12),
                                       (I.gnp(100, 2.4 / 100, 100), 0), (I.gnp(200, 1.9 / 200, 200), 0),
                                       (I.complete_bipartite(8, 8), 0)],
                         ids=lambda x: getattr(x, "name", str(x)))
def test_noalloc_matches_enumerate_twice(cc, g, max_len):
    with cc.Context(frontier_bytes=1 << 30) as ctx:
        ref = ctx.enumerate(g, max_len=max_len)
    for _ in range(2):  # two calls in a row share (and must clear) the fixed array
        s, hist, h, tc = _noalloc(cc, g, max_len)
        assert s == cc.CC_OK, cc.status_str(s)
        assert hist.tolist() == ref.hist.tolist()
        assert h == ref.hash
        assert tc.tolist() == ref.tcount.tolist()


def test_noalloc_rejects_too_large(cc):
    s, *_ = _noalloc(cc, I.cycle(257))
    assert s == cc.CC_ERR_UNSUPPORTED


def test_noalloc_rejects_unsorted_rows(cc):
    g = I.grid(3, 3)
    rp, cl = g.row_ptr.copy(), g.col.copy()
    cl[rp[4]:rp[5]] = cl[rp[4]:rp[5]][::-1]
    s, *_ = _noalloc(cc, I.Graph(g.n, rp, cl))
    assert s == cc.CC_ERR_INVALID_GRAPH


def test_noalloc_chunks_a_frontier_larger_than_the_array(cc):
    # the 8 x 8 grid's two largest levels hold about 5.7 M paths (over 100 MB of records),
    # more than the array's frontier: the expansion must go depth-first in chunks.  A
    # context with a frontier of the array's size shows that such a run spills.
    g = I.grid(8, 8)
    with cc.Context(frontier_bytes=63 << 20) as ctx:
        assert ctx.enumerate(g).info.spilled == 1
    ref = oracle.enumerate_cycles(g)
    for _ in range(2):
        s, hist, h, tc = _noalloc(cc, g)
        assert s == cc.CC_OK, cc.status_str(s)
        assert hist.tolist() == ref.hist.tolist() and h == ref.hash and tc.tolist() == ref.tcount.tolist()


def test_noalloc_capacity_error_then_recovers(cc):
    # K_{128,128}: its initial triplets (up to 127 * 16384 / 2) need more than half of the
    # array; the call fails cleanly and the next call is exact
    s, *_ = _noalloc(cc, I.complete_bipartite(128, 128))
    assert s == cc.CC_ERR_CAPACITY
    g = I.gnp(60, 0.15, 7)
    ref = oracle.enumerate_cycles(g)
    s, hist, h, tc = _noalloc(cc, g)
    assert s == cc.CC_OK and hist.tolist() == ref.hist.tolist() and h == ref.hash


def test_noalloc_rejects_bogus_offsets(cc):
    # row_ptr[n] beyond n (n - 1) is refused before col_idx is read
    g = I.grid(3, 3)
    rp = g.row_ptr.copy()
    rp[-1] = 9 * 8 + 1
    s, *_ = _noalloc(cc, I.Graph(g.n, rp, g.col))
    assert s == cc.CC_ERR_INVALID_GRAPH
