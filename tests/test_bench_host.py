"""Host-side logic of bench.py (no GPU): the reading of a per-step trace into the levels
that two-level steps expanded without storing, and the algorithmic bytes that follow."""
import importlib.util
import os
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_unstored_levels_from_trace():
    b = _bench()
    tc = np.array([0, 0, 0, 5, 7, 9, 4, 0], dtype=np.uint64)
    assert b.unstored_levels(tc, [5, 7, 9, 4]) == set()      # one level per step
    assert b.unstored_levels(tc, [5, 16, 4]) == {5}          # t=4 step also expanded t=5
    assert b.unstored_levels(tc, [12, 13]) == {4, 6}
    assert b.unstored_levels(tc, [3, 2, 7, 9, 4]) == set()   # chunked steps: not resolved
    assert b.unstored_levels(tc, [5, 7]) == set()            # incomplete trace


def test_algorithmic_bytes_counts_stored_levels():
    b = _bench()
    tc = np.array([0, 0, 0, 5, 7, 9, 4, 0], dtype=np.uint64)
    bitset = SimpleNamespace(tcount=tc, info=SimpleNamespace(mode=1))
    # 20-byte records: every stored path read once, every one after the triplets written once
    assert b.algorithmic_bytes(bitset, 60) == 20 * (2 * 25 - 5)
    assert b.algorithmic_bytes(bitset, 60, {5}) == 20 * (2 * 16 - 5)
    assert b.algorithmic_bytes(bitset, 100) == 28 * (2 * 25 - 5)
    csr = SimpleNamespace(tcount=tc, info=SimpleNamespace(mode=2))
    # u16 ids padded to 8: 16 bytes for t <= 8
    assert b.algorithmic_bytes(csr, 2000) == 16 * 2 * 25 - 16 * 5
