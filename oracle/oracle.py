"""ctypes wrapper of the C oracle ``cc_oracle.c`` (test infrastructure only).

Functions mirror the C entry points: degree labelling (Section 2), Algorithm 1
(``enumerate_cycles``) and the subset brute force of the definition (``bruteforce``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cc_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libccoracle.so")
_lib = None
_lock = threading.Lock()

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no target-specific flags)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.cco_vertex_hash.restype = ctypes.c_uint64
            lib.cco_vertex_hash.argtypes = [ctypes.c_uint32]
            lib.cco_cycle_hash.restype = ctypes.c_uint64
            lib.cco_cycle_hash.argtypes = [_u32p, ctypes.c_uint32]
            lib.cco_splitmix64_next.restype = ctypes.c_uint64
            lib.cco_splitmix64_next.argtypes = [_u64p]
            lib.cco_degree_labeling.restype = None
            lib.cco_degree_labeling.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u32p]
            lib.cco_enumerate.restype = ctypes.c_int
            lib.cco_enumerate.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint32,
                                          ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p, _u64p,
                                          _u32p, _u64p, ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p]
            lib.cco_bruteforce.restype = ctypes.c_int
            lib.cco_bruteforce.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint32, _u64p, _u64p,
                                           _u32p, _u64p, ctypes.c_uint64, ctypes.c_uint64, _u64p, _u64p]
            lib.cco_niche_overlap.restype = ctypes.c_uint64
            lib.cco_niche_overlap.argtypes = [ctypes.c_uint32, _u32p, _u32p, _u32p, _u32p]
            lib.cco_triplet_count.restype = ctypes.c_uint64
            lib.cco_triplet_count.argtypes = [ctypes.c_uint32, _u32p, _u32p]
            _lib = lib
    return _lib


def _p32(a):
    return a.ctypes.data_as(_u32p)


def _p64(a):
    return a.ctypes.data_as(_u64p)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint32)
    cl = np.ascontiguousarray(g.col, dtype=np.uint32)
    if cl.size == 0:
        cl = np.zeros(1, dtype=np.uint32)
    return rp, cl


def effective_len(n: int, max_len: int) -> int:
    return n if (max_len == 0 or max_len > n) else max_len


@dataclass
class Result:
    hist: np.ndarray            # uint64 [L'+1]; hist[k] = chordless cycles with k vertices
    hash: int                   # sum of per-cycle hashes mod 2^64
    tcount: Optional[np.ndarray]  # uint64 [L'+1]; paths of t vertices placed in T (Algorithm 1 only)
    cycles: Optional[List[tuple]]  # canonical ordered cycles, if requested

    @property
    def total(self) -> int:
        return int(self.hist.sum())


def vertex_hash(v: int) -> int:
    return int(_load().cco_vertex_hash(v))


def cycle_hash(c) -> int:
    a = np.ascontiguousarray(c, dtype=np.uint32)
    return int(_load().cco_cycle_hash(_p32(a), a.size))


def splitmix64_next(state: int):
    s = ctypes.c_uint64(state)
    out = _load().cco_splitmix64_next(ctypes.byref(s))
    return int(out), int(s.value)


def degree_labeling(g) -> np.ndarray:
    rp, cl = _csr(g)
    lab = np.zeros(max(g.n, 1), dtype=np.uint32)
    _load().cco_degree_labeling(g.n, _p32(rp), _p32(cl), _p32(lab))
    return lab[: g.n]


def triplet_count(g) -> int:
    rp, cl = _csr(g)
    return int(_load().cco_triplet_count(g.n, _p32(rp), _p32(cl)))


def _cycles_from(offs, verts, count):
    return [tuple(int(x) for x in verts[offs[i]:offs[i + 1]]) for i in range(count)]


def enumerate_cycles(g, max_len: int = 0, cycles: bool = False, part: int = 0, nparts: int = 1) -> Result:
    """Algorithm 1 over the whole graph (or over the triplets of one part)."""
    lib = _load()
    rp, cl = _csr(g)
    L = effective_len(g.n, max_len)
    hist = np.zeros(L + 1, dtype=np.uint64)
    tcount = np.zeros(L + 1, dtype=np.uint64)
    h = ctypes.c_uint64(0)
    nc = ctypes.c_uint64(0)
    nv = ctypes.c_uint64(0)
    if not cycles:
        rc = lib.cco_enumerate(g.n, _p32(rp), _p32(cl), max_len, part, nparts, _p64(hist), ctypes.byref(h),
                               _p64(tcount), None, None, 0, 0, ctypes.byref(nc), ctypes.byref(nv))
        if rc != 0:
            raise MemoryError("oracle allocation failed")
        return Result(hist, int(h.value), tcount, None)
    cap_c, cap_v = 1024, 8192
    while True:
        offs = np.zeros(cap_c + 1, dtype=np.uint64)
        verts = np.zeros(cap_v, dtype=np.uint32)
        rc = lib.cco_enumerate(g.n, _p32(rp), _p32(cl), max_len, part, nparts, _p64(hist), ctypes.byref(h),
                               _p64(tcount), _p32(verts), _p64(offs), cap_c, cap_v, ctypes.byref(nc), ctypes.byref(nv))
        if rc != 0:
            raise MemoryError("oracle allocation failed")
        if nc.value <= cap_c and nv.value <= cap_v:
            return Result(hist, int(h.value), tcount, _cycles_from(offs, verts, nc.value))
        cap_c, cap_v = max(cap_c, nc.value), max(cap_v, nv.value)


def bruteforce(g, max_len: int = 0, cycles: bool = False) -> Result:
    """Every vertex subset tested against the definition (n <= 30)."""
    lib = _load()
    if g.n > 30:
        raise ValueError("brute force needs n <= 30")
    rp, cl = _csr(g)
    L = effective_len(g.n, max_len)
    hist = np.zeros(L + 1, dtype=np.uint64)
    h = ctypes.c_uint64(0)
    nc = ctypes.c_uint64(0)
    nv = ctypes.c_uint64(0)
    cap_c, cap_v = (1024, 8192) if cycles else (0, 0)
    while True:
        offs = np.zeros(cap_c + 1, dtype=np.uint64)
        verts = np.zeros(max(cap_v, 1), dtype=np.uint32)
        rc = lib.cco_bruteforce(g.n, _p32(rp), _p32(cl), max_len, _p64(hist), ctypes.byref(h),
                                _p32(verts) if cycles else None, _p64(offs) if cycles else None,
                                cap_c, cap_v, ctypes.byref(nc), ctypes.byref(nv))
        if rc != 0:
            raise ValueError("brute force refused")
        if not cycles:
            return Result(hist, int(h.value), None, None)
        if nc.value <= cap_c and nv.value <= cap_v:
            return Result(hist, int(h.value), None, _cycles_from(offs, verts, nc.value))
        cap_c, cap_v = max(cap_c, nc.value), max(cap_v, nv.value)


def enumerate_parallel(g, max_len: int = 0, threads: int = 0) -> Result:
    """Algorithm 1 split over the initial triplets (index modulo ``threads``) and run on a
    thread pool; ctypes releases the GIL during each call.  Sums the parts."""
    import concurrent.futures as cf
    threads = threads or os.cpu_count() or 1
    with cf.ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda p: enumerate_cycles(g, max_len, part=p, nparts=threads), range(threads)))
    hist = sum(p.hist for p in parts)
    tcount = sum(p.tcount for p in parts)
    return Result(hist, sum(p.hash for p in parts) % (1 << 64), tcount, None)


def niche_overlap(n: int, prey_ptr, prey_idx):
    """Niche overlap graph of a food web by its definition (Section 5): (row_ptr, col)."""
    rp = np.ascontiguousarray(prey_ptr, dtype=np.uint32)
    pi = np.ascontiguousarray(prey_idx if len(prey_idx) else [0], dtype=np.uint32)
    out_rp = np.zeros(n + 1, dtype=np.uint32)
    out_col = np.zeros(max(n * (n - 1), 1), dtype=np.uint32)
    nnz = int(_load().cco_niche_overlap(n, _p32(rp), _p32(pi), _p32(out_rp), _p32(out_col)))
    return out_rp, out_col[:nnz].copy()
