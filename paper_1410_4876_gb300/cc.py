"""ctypes binding of the C ABI in ``include/cc.h`` (argument marshalling only).

The functions keep the C names (``cc_context_create``, ``cc_graph_load``, ``cc_enumerate``,
``cc_batch_submit``, ``cc_batch_poll`` ...).  Every step of the enumeration runs in the
CUDA library; this module only converts numpy arrays to pointers.  There is no CPU
fallback: if the library is missing, loading it raises.

PyTorch is used for plumbing only: ``Context(use_torch=True)`` hands the library a
frontier arena allocated by torch's caching allocator and torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcc.so")

CC_OK = 0
CC_PENDING = 1
CC_ERR_ARG = -1
CC_ERR_INVALID_GRAPH = -2
CC_ERR_OOM = -3
CC_ERR_CUDA = -4
CC_ERR_TIMEOUT = -5
CC_ERR_TRUNCATED = -6
CC_ERR_UNSUPPORTED = -7
CC_ERR_CAPACITY = -8

CC_MODE_AUTO = 0
CC_MODE_BITSET = 1
CC_MODE_CSR = 2

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_dblp = ctypes.POINTER(ctypes.c_double)


class cc_options(ctypes.Structure):
    _fields_ = [
        ("frontier_bytes", ctypes.c_uint64),
        ("stream", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_uint64),
        ("threads_per_block", ctypes.c_uint32),
        ("blocks_per_sm", ctypes.c_uint32),
        ("mode", ctypes.c_uint32),
        ("spin_limit", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("paths_per_thread", ctypes.c_uint32),
        ("small_phase_paths", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("host_frontier_bytes", ctypes.c_uint64),
    ]


CC_FLAG_NO_CLUSTER_PHASE = 1
CC_FLAG_NO_GRAPH = 2
CC_FLAG_NO_FUSE = 4


class cc_limits(ctypes.Structure):
    _fields_ = [
        ("max_n_bitset", ctypes.c_uint32),
        ("max_n_csr", ctypes.c_uint32),
        ("max_n_batch", ctypes.c_uint32),
        ("max_batch", ctypes.c_uint32),
    ]


class cc_run_info(ctypes.Structure):
    _fields_ = [
        ("ms_proc", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("ms_engine", ctypes.c_double),
        ("steps", ctypes.c_uint64),
        ("paths", ctypes.c_uint64),
        ("cycles", ctypes.c_uint64),
        ("mode", ctypes.c_uint32),
        ("grid_blocks", ctypes.c_uint32),
        ("spilled", ctypes.c_uint32),
        ("launches", ctypes.c_uint32),
        ("peak_bytes", ctypes.c_uint64),
        ("dev_error", ctypes.c_int32),
        ("dev_error_info", ctypes.c_int32),
        ("replayed", ctypes.c_uint32),
        ("host_offloads", ctypes.c_uint32),
    ]


class cc_tune_result(ctypes.Structure):
    _fields_ = [
        ("best", cc_options),
        ("ms_best", ctypes.c_double),
        ("ms_default", ctypes.c_double),
        ("candidates", ctypes.c_uint32),
        ("from_cache", ctypes.c_uint32),
        ("graph_class", ctypes.c_char * 64),
    ]


class cc_cycles(ctypes.Structure):
    _fields_ = [
        ("capacity_cycles", ctypes.c_uint64),
        ("capacity_vertices", ctypes.c_uint64),
        ("offsets", _u64p),
        ("vertices", _u32p),
        ("count", ctypes.c_uint64),
        ("total_vertices", ctypes.c_uint64),
    ]


class CCError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})" if what else f"{status_str(status)} ({status})")


_lib = None

# exported symbols and their ctypes signatures (the C names of include/cc.h)
SIGNATURES = {
    "cc_context_create": (ctypes.c_int32, [ctypes.POINTER(cc_options), ctypes.POINTER(ctypes.c_void_p)]),
    "cc_context_destroy": (None, [ctypes.c_void_p]),
    "cc_status_str": (ctypes.c_char_p, [ctypes.c_int32]),
    "cc_get_limits": (None, [ctypes.POINTER(cc_limits)]),
    "cc_graph_load": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, _u32p, _u32p, ctypes.POINTER(ctypes.c_void_p)]),
    "cc_graph_free": (None, [ctypes.c_void_p]),
    "cc_graph_info": (ctypes.c_int32, [ctypes.c_void_p, _u32p, _u64p, _u32p]),
    "cc_enumerate": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, _u64p, _u64p, _u64p,
                                      ctypes.POINTER(cc_cycles), ctypes.POINTER(cc_run_info)]),
    "cc_enumerate_part": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                           _u64p, _u64p, _u64p, ctypes.POINTER(cc_cycles),
                                           ctypes.POINTER(cc_run_info)]),
    "cc_batch_submit": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, _u32p, _u64p, _u32p, _u64p, _u32p,
                                         ctypes.c_uint32, _u64p]),
    "cc_batch_load": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, _u32p, _u64p, _u32p, _u64p, _u32p,
                                       ctypes.POINTER(ctypes.c_void_p), _u32p]),
    "cc_batch_run": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, _u64p]),
    "cc_batch_free": (None, [ctypes.c_void_p]),
    "cc_batch_poll": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, _u64p, ctypes.c_uint32,
                                       _u64p, _u64p, _dblp, ctypes.POINTER(cc_run_info)]),
    "cc_get_trace": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, _u64p, _u64p, _u64p]),
    "cc_enumerate_stream": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                             ctypes.c_void_p, ctypes.c_void_p, _u64p, _u64p, _u64p, _u32p,
                                             ctypes.POINTER(cc_run_info)]),
    "cc_context_set_options": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(cc_options)]),
    "cc_tune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_char_p, ctypes.POINTER(cc_tune_result)]),
    "cc_tune_batch": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, _u32p, _u64p, _u32p, _u64p, _u32p,
                                       ctypes.c_uint32, ctypes.c_char_p, ctypes.POINTER(cc_tune_result)]),
    "cc_niche_overlap": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, _u32p, _u32p, _u32p, _u32p,
                                          ctypes.c_uint64, _u64p]),
    "cc_enumerate_noalloc": (ctypes.c_int32, [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint32, ctypes.c_void_p,
                                              _u64p, _u64p, _u64p]),
}


def load_library(path: Optional[str] = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_str(s: int) -> str:
    try:
        return load_library().cc_status_str(s).decode()
    except ImportError:
        return str(s)


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_u32p)


def _p64(a: np.ndarray):
    return a.ctypes.data_as(_u64p)


def _check(s: int, what: str):
    if s != CC_OK:
        raise CCError(s, what)


def cc_get_limits() -> cc_limits:
    lim = cc_limits()
    load_library().cc_get_limits(ctypes.byref(lim))
    return lim


def cc_context_create(opts: Optional[cc_options] = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().cc_context_create(ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)),
           "cc_context_create")
    return h


def cc_context_destroy(ctx) -> None:
    load_library().cc_context_destroy(ctx)


def cc_context_set_options(ctx, opts: cc_options) -> int:
    return load_library().cc_context_set_options(ctx, ctypes.byref(opts))


def _path_arg(path: Optional[str]):
    return os.fsencode(path) if path else None


def cc_tune(g, max_len: int = 0, cache_path: Optional[str] = None):
    """Returns (status, cc_tune_result)."""
    out = cc_tune_result()
    s = load_library().cc_tune(g, max_len, _path_arg(cache_path), ctypes.byref(out))
    return s, out


def cc_tune_batch(ctx, graphs: Sequence, max_len: int = 0, cache_path: Optional[str] = None):
    """Returns (status, cc_tune_result)."""
    from .inputs import pack
    ns, row_off, rp, col_off, cl = pack(graphs)
    if cl.size == 0:
        cl = np.zeros(1, dtype=np.uint32)
    out = cc_tune_result()
    s = load_library().cc_tune_batch(ctx, len(graphs), _p32(ns), _p64(row_off), _p32(rp), _p64(col_off), _p32(cl),
                                     max_len, _path_arg(cache_path), ctypes.byref(out))
    return s, out


def cc_graph_load(ctx, n: int, row_ptr: np.ndarray, col_idx: np.ndarray):
    rp = np.ascontiguousarray(row_ptr, dtype=np.uint32)
    cl = np.ascontiguousarray(col_idx, dtype=np.uint32)
    if cl.size == 0:
        cl = np.zeros(1, dtype=np.uint32)
    h = ctypes.c_void_p()
    s = load_library().cc_graph_load(ctx, n, _p32(rp), _p32(cl), ctypes.byref(h))
    return s, h


def cc_graph_free(g) -> None:
    load_library().cc_graph_free(g)


def cc_enumerate(g, n: int, max_len: int = 0, tcount: bool = True, cycles_capacity: Optional[tuple] = None,
                 part: int = 0, nparts: int = 1):
    """Returns (status, hist, hash, tcount, cycles, info); cycles is a list of tuples or None.
    nparts > 1 calls cc_enumerate_part (this part of the initial triplets only)."""
    L = n if (max_len == 0 or max_len > n) else max_len
    hist = np.zeros(L + 1, dtype=np.uint64)
    tc = np.zeros(L + 1, dtype=np.uint64) if tcount else None
    hsh = ctypes.c_uint64(0)
    info = cc_run_info()
    cyc = None
    offs = verts = None
    if cycles_capacity is not None:
        cap_c, cap_v = cycles_capacity
        offs = np.zeros(cap_c + 1, dtype=np.uint64)
        verts = np.zeros(max(cap_v, 1), dtype=np.uint32)
        cyc = cc_cycles(cap_c, cap_v, _p64(offs), _p32(verts), 0, 0)
    if nparts != 1 or part:
        s = load_library().cc_enumerate_part(g, max_len, part, nparts, _p64(hist), ctypes.byref(hsh),
                                             _p64(tc) if tc is not None else None,
                                             ctypes.byref(cyc) if cyc is not None else None, ctypes.byref(info))
    else:
        s = load_library().cc_enumerate(g, max_len, _p64(hist), ctypes.byref(hsh),
                                        _p64(tc) if tc is not None else None,
                                        ctypes.byref(cyc) if cyc is not None else None, ctypes.byref(info))
    out_cycles = None
    if cyc is not None:
        if s == CC_OK:
            out_cycles = [tuple(int(x) for x in verts[offs[i]:offs[i + 1]]) for i in range(cyc.count)]
        elif s == CC_ERR_TRUNCATED:
            out_cycles = (int(cyc.count), int(cyc.total_vertices))
    return s, hist, int(hsh.value), tc, out_cycles, info


# void sink(void* user, uint64_t count, const uint64_t* starts, const uint32_t* lengths,
#           const uint32_t* vertices, uint64_t total_vertices)
CYCLE_SINK = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, _u64p, _u32p, _u32p, ctypes.c_uint64)


def cc_enumerate_stream(g, n: int, sink, max_len: int = 0, chunk_cycles: int = 1 << 20,
                        chunk_vertices: int = 1 << 24):
    """Streamed cycle list.  ``sink(starts, lengths, vertices)`` receives each round's
    cycles as numpy views (valid during the call only): cycle i is
    vertices[starts[i]:starts[i] + lengths[i]].  Returns (status, hist, hash, tcount,
    rounds, info)."""
    L = n if (max_len == 0 or max_len > n) else max_len
    hist = np.zeros(L + 1, dtype=np.uint64)
    tc = np.zeros(L + 1, dtype=np.uint64)
    hsh = ctypes.c_uint64(0)
    rounds = ctypes.c_uint32(0)
    info = cc_run_info()
    err = []

    def _sink(user, count, starts, lengths, vertices, nv):
        try:
            sink(np.ctypeslib.as_array(starts, (count,)), np.ctypeslib.as_array(lengths, (count,)),
                 np.ctypeslib.as_array(vertices, (nv,)))
        except BaseException as x:  # an exception cannot cross the C frame: re-raised below
            err.append(x)

    cb = CYCLE_SINK(_sink)
    s = load_library().cc_enumerate_stream(g, max_len, chunk_cycles, chunk_vertices, ctypes.cast(cb, ctypes.c_void_p),
                                           None, _p64(hist), ctypes.byref(hsh), _p64(tc), ctypes.byref(rounds),
                                           ctypes.byref(info))
    if err:
        raise err[0]
    return s, hist, int(hsh.value), tc, int(rounds.value), info


def cc_batch_submit(ctx, graphs: Sequence, max_len: int = 0):
    from .inputs import pack
    ns, row_off, rp, col_off, cl = pack(graphs)
    if cl.size == 0:
        cl = np.zeros(1, dtype=np.uint32)
    bid = ctypes.c_uint64(0)
    s = load_library().cc_batch_submit(ctx, len(graphs), _p32(ns), _p64(row_off), _p32(rp), _p64(col_off), _p32(cl),
                                       max_len, ctypes.byref(bid))
    return s, int(bid.value)


def cc_niche_overlap(ctx, n: int, prey_ptr, prey_idx, col_capacity: Optional[int] = None):
    """Niche overlap graph of a food web: (status, row_ptr, col).  With col_capacity None
    the call is made twice (sizes, then ids)."""
    pp = np.ascontiguousarray(prey_ptr, dtype=np.uint32)
    pi = np.ascontiguousarray(prey_idx if len(prey_idx) else np.zeros(1), dtype=np.uint32)
    rp = np.zeros(n + 1, dtype=np.uint32)
    nnz = ctypes.c_uint64(0)
    cap = 0 if col_capacity is None else col_capacity
    col = np.zeros(max(cap, 1), dtype=np.uint32)
    s = load_library().cc_niche_overlap(ctx, n, _p32(pp), _p32(pi), _p32(rp), _p32(col), cap, ctypes.byref(nnz))
    if s == CC_ERR_TRUNCATED and col_capacity is None:
        cap = int(nnz.value)
        col = np.zeros(max(cap, 1), dtype=np.uint32)
        s = load_library().cc_niche_overlap(ctx, n, _p32(pp), _p32(pi), _p32(rp), _p32(col), cap, ctypes.byref(nnz))
    return s, rp, col[:int(nnz.value)]


def cc_batch_load(ctx, packed):
    """packed = (n, row_off, row_ptr, col_off, col_idx) as made by inputs.pack; returns
    (status, set handle, index of the first bad graph)."""
    ns, row_off, rp, col_off, cl = packed
    if cl.size == 0:
        cl = np.zeros(1, dtype=np.uint32)
    h = ctypes.c_void_p(None)
    bad = ctypes.c_uint32(0)
    s = load_library().cc_batch_load(ctx, ns.size, _p32(ns), _p64(row_off), _p32(rp), _p64(col_off), _p32(cl),
                                     ctypes.byref(h), ctypes.byref(bad))
    return s, h.value, int(bad.value)


def cc_batch_run(bset, max_len: int = 0):
    bid = ctypes.c_uint64(0)
    s = load_library().cc_batch_run(bset, max_len, ctypes.byref(bid))
    return s, int(bid.value)


def cc_batch_free(bset) -> None:
    load_library().cc_batch_free(bset)


def cc_batch_poll(ctx, batch: int, count: int, timeout_us: int = 0, hist_stride: int = 65):
    hist = np.zeros((count, hist_stride), dtype=np.uint64)
    hsh = np.zeros(count, dtype=np.uint64)
    paths = np.zeros(count, dtype=np.uint64)
    done = np.zeros(count, dtype=np.float64)
    info = cc_run_info()
    s = load_library().cc_batch_poll(ctx, batch, timeout_us, _p64(hist), hist_stride, _p64(hsh), _p64(paths),
                                     done.ctypes.data_as(_dblp), ctypes.byref(info))
    return s, hist, hsh, paths, done, info


# ------------------------------------------------------------------ convenience layer

@dataclass
class Result:
    hist: np.ndarray
    hash: int
    tcount: Optional[np.ndarray]
    cycles: Optional[List[tuple]]
    info: cc_run_info

    @property
    def total(self) -> int:
        return int(self.hist.sum())

    @property
    def paths(self) -> int:
        return int(self.tcount.sum()) if self.tcount is not None else int(self.info.paths)


class Context:
    """Owns a cc_context.  With ``use_torch`` the frontier arena comes from torch's
    caching allocator and the work runs on torch's current stream."""

    def __init__(self, frontier_bytes: int = 0, mode: int = CC_MODE_AUTO, threads_per_block: int = 0,
                 blocks_per_sm: int = 0, spin_limit: int = 0, use_torch: bool = False, stream: int = 0,
                 flags: int = 0, paths_per_thread: int = 0, small_phase_paths: int = 0,
                 host_frontier_bytes: int = 0):
        self._ws = None
        opts = cc_options()
        opts.frontier_bytes = frontier_bytes
        opts.mode = mode
        opts.threads_per_block = threads_per_block
        opts.blocks_per_sm = blocks_per_sm
        opts.spin_limit = spin_limit
        opts.stream = stream or None
        opts.flags = flags
        opts.paths_per_thread = paths_per_thread
        opts.small_phase_paths = small_phase_paths
        opts.host_frontier_bytes = host_frontier_bytes
        if use_torch:
            import torch
            nbytes = frontier_bytes or (1 << 30)
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            opts.workspace = self._ws.data_ptr()
            opts.workspace_bytes = nbytes
            opts.stream = torch.cuda.current_stream().cuda_stream
        self.handle = cc_context_create(opts)

    def close(self):
        if getattr(self, "handle", None):
            cc_context_destroy(self.handle)
            self.handle = None
        self._ws = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, opts: cc_options) -> None:
        _check(cc_context_set_options(self.handle, opts), "cc_context_set_options")

    def tune_batch(self, graphs: Sequence, max_len: int = 0, cache_path: Optional[str] = None) -> cc_tune_result:
        s, out = cc_tune_batch(self.handle, graphs, max_len, cache_path)
        _check(s, "cc_tune_batch")
        return out

    def load(self, graph) -> "LoadedGraph":
        s, h = cc_graph_load(self.handle, graph.n, graph.row_ptr, graph.col)
        _check(s, "cc_graph_load")
        return LoadedGraph(self, h, graph.n)

    def enumerate(self, graph, max_len: int = 0, cycles: bool = False) -> Result:
        with self.load(graph) as g:
            return g.enumerate(max_len, cycles)

    def batch(self, graphs: Sequence, max_len: int = 0, timeout_s: float = 600.0):
        """Submit a batch and wait for it; returns (hist[count, 65], hash[count], paths[count],
        done_us[count], info)."""
        s, bid = cc_batch_submit(self.handle, graphs, max_len)
        _check(s, "cc_batch_submit")
        return _wait_batch(self, bid, len(graphs), timeout_s)


    def load_batch(self, graphs: Sequence) -> "BatchSet":
        from .inputs import pack
        s, h, bad = cc_batch_load(self.handle, pack(graphs))
        _check(s, f"cc_batch_load (graph {bad})")
        return BatchSet(self, h, len(graphs))


def _wait_batch(ctx: "Context", bid: int, count: int, timeout_s: float):
    import time
    t_end = time.time() + timeout_s
    while True:
        s, hist, hsh, paths, done, info = cc_batch_poll(ctx.handle, bid, count, 200000)
        if s != CC_PENDING:
            break
        if time.time() > t_end:
            raise CCError(CC_ERR_TIMEOUT, "cc_batch_poll")
    _check(s, "cc_batch_poll")
    return hist, hsh, paths, done, info


class BatchSet:
    """Graphs resident on the device for repeated batched enumeration (cc_batch_load)."""

    def __init__(self, ctx: Context, handle, count: int):
        self.ctx, self.handle, self.count = ctx, handle, count

    def run(self, max_len: int = 0, timeout_s: float = 600.0):
        """cc_batch_run + cc_batch_poll: (hist[count, 65], hash[count], paths[count],
        done_us[count], info)."""
        s, bid = cc_batch_run(self.handle, max_len)
        _check(s, "cc_batch_run")
        return _wait_batch(self.ctx, bid, self.count, timeout_s)

    def close(self):
        if getattr(self, "handle", None):
            cc_batch_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class LoadedGraph:
    def __init__(self, ctx: Context, handle, n: int):
        self.ctx, self.handle, self.n = ctx, handle, n

    def enumerate(self, max_len: int = 0, cycles: bool = False, part: int = 0, nparts: int = 1) -> Result:
        cap = (1024, 8192) if cycles else None
        while True:
            s, hist, h, tc, cyc, info = cc_enumerate(self.handle, self.n, max_len, True, cap, part, nparts)
            if cycles and s == CC_ERR_TRUNCATED:
                cap = (int(cyc[0]) + 16, int(cyc[1]) + 64)
                continue
            _check(s, "cc_enumerate")
            return Result(hist, h, tc, cyc, info)

    def enumerate_stream(self, sink, max_len: int = 0, chunk_cycles: int = 1 << 20,
                         chunk_vertices: int = 1 << 24):
        """Every cycle through ``sink(starts, lengths, vertices)``, round by round (see
        cc_enumerate_stream); returns (Result without cycles, rounds)."""
        s, hist, h, tc, rounds, info = cc_enumerate_stream(self.handle, self.n, sink, max_len, chunk_cycles,
                                                           chunk_vertices)
        _check(s, "cc_enumerate_stream")
        return Result(hist, h, tc, None, info), rounds

    def tune(self, max_len: int = 0, cache_path: Optional[str] = None) -> cc_tune_result:
        s, out = cc_tune(self.handle, max_len, cache_path)
        _check(s, "cc_tune")
        return out

    def close(self):
        if self.handle:
            cc_graph_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def cc_get_trace(ctx, cap: int = 1 << 16):
    """Per-step trace of the last cc_enumerate: (t_ns[steps], expanded[steps])."""
    t = np.zeros(cap, dtype=np.uint64)
    e = np.zeros(cap, dtype=np.uint64)
    n = ctypes.c_uint64(0)
    _check(load_library().cc_get_trace(ctx, cap, _p64(t), _p64(e), ctypes.byref(n)), "cc_get_trace")
    k = min(int(n.value), cap)
    return t[:k], e[:k]


# ------------------------------------------------------------------ serving

class cc_serve_options(ctypes.Structure):
    _fields_ = [
        ("slots", ctypes.c_uint32),
        ("max_len", ctypes.c_uint32),
        ("admit_bytes", ctypes.c_uint64),
        ("steps_per_round", ctypes.c_uint32),
        ("pad", ctypes.c_uint32),
        ("reserve_paths", ctypes.c_uint64),
    ]


class cc_completion(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_uint64),
        ("hash", ctypes.c_uint64),
        ("total", ctypes.c_uint64),
        ("paths", ctypes.c_uint64),
        ("hist", ctypes.c_uint64 * 65),
        ("wait_us", ctypes.c_double),
        ("latency_us", ctypes.c_double),
    ]


SIGNATURES.update({
    "cc_serve_create": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(cc_serve_options),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "cc_serve_destroy": (None, [ctypes.c_void_p]),
    "cc_serve_submit": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint64, _u64p]),
    "cc_serve_step": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(cc_completion), ctypes.c_uint32,
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(ctypes.c_uint32)]),
    "cc_serve_predict_bytes": (ctypes.c_uint64, [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]),
})


def cc_serve_predict_bytes(n: int, m: int, max_degree: int) -> int:
    return int(load_library().cc_serve_predict_bytes(n, m, max_degree))


class Server:
    """Continuous-batching request loop on a context (see cc_serve_* in include/cc.h)."""

    def __init__(self, ctx: Context, slots: int = 0, max_len: int = 0, admit_bytes: int = 0,
                 steps_per_round: int = 0, reserve_paths: int = 0, cap: int = 4096):
        o = cc_serve_options(slots, max_len, admit_bytes, steps_per_round, 0, reserve_paths)
        self.handle = ctypes.c_void_p()
        _check(load_library().cc_serve_create(ctx.handle, ctypes.byref(o), ctypes.byref(self.handle)),
               "cc_serve_create")
        self._buf = (cc_completion * cap)()
        self._cap = cap

    def submit(self, graph, predicted_bytes: int = 0) -> int:
        rp = np.ascontiguousarray(graph.row_ptr, dtype=np.uint32)
        cl = np.ascontiguousarray(graph.col if graph.col.size else np.zeros(1, np.uint32), dtype=np.uint32)
        rid = ctypes.c_uint64(0)
        _check(load_library().cc_serve_submit(self.handle, graph.n, _p32(rp), _p32(cl), predicted_bytes,
                                              ctypes.byref(rid)), "cc_serve_submit")
        return int(rid.value)

    def step(self):
        """One round; returns (completions, in_flight, queued).  Each completion is a dict."""
        n = ctypes.c_uint32(0)
        inf = ctypes.c_uint32(0)
        q = ctypes.c_uint32(0)
        _check(load_library().cc_serve_step(self.handle, self._buf, self._cap, ctypes.byref(n), ctypes.byref(inf),
                                            ctypes.byref(q)), "cc_serve_step")
        out = []
        for i in range(n.value):
            c = self._buf[i]
            out.append({"id": int(c.id), "hash": int(c.hash), "total": int(c.total), "paths": int(c.paths),
                        "hist": np.array(c.hist[:], dtype=np.uint64), "wait_us": c.wait_us,
                        "latency_us": c.latency_us})
        return out, int(inf.value), int(q.value)

    def close(self):
        if getattr(self, "handle", None):
            load_library().cc_serve_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
