"""Benchmark: chordless cycles/s and paths expanded/s on one GB300; batched against
per-graph launches; per-graph p50/p99.

Default workload (one step): the 4096-graph batch mixture (seed 0: 50% G(n,p) with n in
[16,64] and p in [0.08,0.3], 30% k x l grids with k,l in [3,6], 20% K_{a,b} with a,b in
[2,8]), every chordless cycle of every graph, enumerated by one persistent launch on
graphs already resident in HBM (cc_batch_load once, then cc_batch_run + cc_batch_poll per
step).  The L2 cache is flushed by a 256 MiB write before every timed step.  The line also
carries, as sub-objects, the single-graph workloads (grid 8x8 + G(60, 0.15, seed 7); G(2000,
4000, seed 11) with cycles of at most 12 vertices) and the serving workload (Poisson
arrivals at 2000/s for 60 s, seed 3), each with its own measurements.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batch|grid8+gnp60|gnm2000|grid6|grid7x10|grid8x10|serve|stream]

--impl reference times the CPU oracle (Algorithm 1 in plain C, test infrastructure) on the
host cores for the same workload and metric, each step a bounded sample.  Under torchrun
(N > 1) every rank runs its own replica of the batch (independent problems, no
collective, weak scaling); for a single-graph workload the ranks split the graph's initial
triplets (cc_enumerate_part) and one all-reduce sums the histograms and hashes.  Rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1410_4876_gb300 import inputs as I  # noqa: E402

METRIC = "chordless cycles/s"
UNIT = "cycles/s"
def batch_desc(count: int) -> str:
    return (f"{count} graphs of the seeded batch mixture (seed 0: 50% G(n,p) n in [16,64] p in [0.08,0.3], "
            "30% k x l grids k,l in [3,6], 20% K_ab a,b in [2,8]); all chordless cycles of every length, "
            "one persistent launch")
WORKLOADS = {
    "grid8+gnp60": ("grid 8x8 (64 vertices, 112 edges, row-major ids) + Erdos-Renyi G(n=60, p=0.15, seed 7); "
                    "all chordless cycles of every length", lambda: [(I.grid(8, 8), 0), (I.gnp(60, 0.15, 7), 0)]),
    "grid6": ("grid 6x6 (36 vertices, 60 edges), all lengths", lambda: [(I.grid(6, 6), 0)]),
    "gnm2000": ("G(n=2000, m=4000, seed 11), cycles up to 12 vertices", lambda: [(I.gnm(2000, 4000, 11), 12)]),
    # the largest synthetic rows of Table 1, for comparison with the paper's own timings
    "grid7x10": ("grid 7x10 (70 vertices, 123 edges), all lengths", lambda: [(I.grid(7, 10), 0)]),
    "grid8x10": ("grid 8x10 (80 vertices, 142 edges), all lengths (Table 1's count-only row)",
                 lambda: [(I.grid(8, 10), 0)]),
}


# ------------------------------------------------------------------ algorithmic bytes

def bitset_record_bytes(W: int) -> int:
    """Per-path record of the bitset forms as the scope table sizes it: W words of blocked
    set plus the path's end ids and length, padded to 16 bytes (16 B for n <= 64)."""
    return 16 * ((8 * W + 4 + 15) // 16)


def csr_record_bytes(t: int) -> int:
    """A CSR path of t vertices: its u16 ids padded to a multiple of 8 (16 B for t <= 8)."""
    return 16 * ((t + 7) // 8)


def algorithmic_bytes(tcount, n: int, mode: int) -> int:
    """Bytes the expansion must move: every stored chordless path (the sets T_t, t = 3 ..
    L'-1, counted in tcount) is written once and read once.  mode 2 = CSR records, else
    bitset records of ceil(n/64) words (1, 2 or 4)."""
    tc = np.asarray(tcount, dtype=np.int64)
    if mode == 2:
        rec = np.array([csr_record_bytes(t) for t in range(tc.size)], dtype=np.int64)
        return int(2 * (tc * rec).sum())
    W = 1 if n <= 64 else (2 if n <= 128 else 4)
    return int(2 * bitset_record_bytes(W) * tc.sum())


# ------------------------------------------------------------------ ranks, clocks, peaks

def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def _dist_init(world):
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group("nccl" if _has_cuda() else "gloo")
    return dist


def max_over_ranks(value: float, dist, device=None) -> float:
    """The largest value over all ranks (the bench times every rank and keeps the slowest)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def steps_for_clocks(steps: int, ms_per_step: float, dist=None, device=None, region_ms: float = 1500.0,
                     cap: int = 5000) -> int:
    """Timed steps for a short workload: at least `steps`, and enough to span about
    `region_ms` so that the 200 ms clock sampler sees the GPU under load several times
    (the same count on every rank)."""
    k = steps
    if ms_per_step > 0:
        k = max(steps, min(cap, int(math.ceil(region_ms / ms_per_step))))
    return int(max_over_ranks(k, dist, device))


def sum_results(hist, hsh: int, dist, device=None):
    """Sum per-rank partial results (histogram, cycle hash mod 2^64) over all ranks: the one
    exchange step of a graph whose initial triplets are split across ranks.  The hash is
    summed as four 16-bit limbs in int64 so that no partial sum overflows."""
    hist = np.asarray(hist, dtype=np.uint64)
    if dist is None:
        return hist, int(hsh) % (1 << 64)
    import torch
    limbs = [(int(hsh) >> (16 * i)) & 0xFFFF for i in range(4)]
    t = torch.tensor(hist.astype(np.int64).tolist() + limbs, dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    v = t.cpu().numpy()
    h = sum(int(v[hist.size + i]) << (16 * i) for i in range(4)) % (1 << 64)
    return v[:hist.size].astype(np.uint64), h


def _has_cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (burst copy)"
    return 6800.0, "fallback"


def _percentiles(x):
    x = np.asarray(x, dtype=np.float64)
    if x.size == 0:
        return None, None
    return float(np.percentile(x, 50)), float(np.percentile(x, 99))


def _frontier_bytes(args, default_mb):
    return (args.frontier_mb or default_mb) << 20


# ------------------------------------------------------------------ committed ncu summaries

_FORM_SOURCES = {"Multi": "cc_expand_multi.cuh", "Bitset": "cc_expand_bitset.cuh", "Csr": "cc_expand_csr.cuh"}


def _engine_fingerprint(kernel: str) -> str:
    """Hash of the code a kernel runs, without comments and whitespace: the persistent
    kernel and planner (cc_engine.cu), the shared helpers (cc_internal.cuh) and the
    expansion form of its record kind (cc_expand_<form>.cuh), so that a committed ncu
    capture is used only for the code it measured, and a change to one form leaves the
    other forms' captures valid."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1410_4876_gb300", "csrc")
    forms = [v for k, v in _FORM_SOURCES.items() if k in kernel] or sorted(_FORM_SOURCES.values())
    text = ""
    for f in ["cc_engine.cu", "cc_internal.cuh"] + forms:
        src = open(os.path.join(csrc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        text += re.sub(r"\s+", "", src)
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def _profile(name: str) -> dict:
    """The committed summary profiles/<name>.json: the kernel's limiter as ncu showed it and
    its DRAM bytes per stored path.  `traffic_per_path` is returned only while the engine
    source matches the capture's fingerprint."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", name + ".json")))
    except Exception:
        return {}
    if d.get("source_fingerprint") != _engine_fingerprint(d.get("kernel", "")):
        d.pop("dram_bytes_per_path", None)
    return d


def roofline(kernel: str, bytes_per_launch: float, ms_per_launch: float, paths_per_launch: float,
             profile: str) -> dict:
    """The dominant kernel against the measured HBM copy bandwidth: algorithmic bytes per
    launch (every stored path written once and read once) over the kernel's average launch
    time from CUDA events on its stream.  `bound` is what the committed ncu capture shows
    limits the kernel; `traffic` is DRAM bytes per launch scaled from that capture by stored
    paths (null when the capture predates the current engine source)."""
    peak, kind = _peaks()
    achieved = bytes_per_launch / (ms_per_launch / 1000.0) / 1e9 if ms_per_launch > 0 else 0.0
    prof = _profile(profile)
    per_path = prof.get("dram_bytes_per_path")
    out = {"bound": prof.get("bound", "hbm"), "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak if peak else None,
           "traffic": per_path * paths_per_launch if per_path else None,
           "kernel": kernel, "peak_kind": kind, "algorithmic_bytes_per_launch": bytes_per_launch,
           "kernel_ms_per_launch": ms_per_launch}
    for k in ("issue_active_pct", "alu_pipe_pct", "dram_throughput_pct", "warps_active_pct"):
        if k in prof:
            out[k] = prof[k]
    if prof:
        out["profile"] = f"profiles/{profile}.md"
    return out


# ------------------------------------------------------------------ CPU oracle (baseline)

def cpu_oracle(items, parts_per_core=2):
    """The oracle as it stands on all host cores: each (graph, max_len) of `items` split
    into parts of its initial triplets (index modulo the part count), the parts run on a
    thread pool (ctypes releases the GIL).  Returns (cycles, paths, seconds, threads)."""
    import concurrent.futures as cf

    import oracle
    cores = os.cpu_count() or 1
    nparts = cores * parts_per_core
    jobs = [(g, L, p) for g, L in items for p in range(nparts)]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(cores) as ex:
        res = list(ex.map(lambda j: oracle.enumerate_cycles(j[0], max_len=j[1], part=j[2], nparts=nparts), jobs))
    dt = time.perf_counter() - t0
    return sum(r.total for r in res), sum(int(r.tcount.sum()) for r in res), dt, cores


def cpu_baseline_line(items, what: str) -> dict:
    c, p, dt, cores = cpu_oracle(items)
    return {"value": c / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what}; triplets split {2 * cores} ways per graph on {cores} threads, {dt:.1f} s",
            "paths_expanded_per_s": p / dt}


def batch_sample(graphs, stride: int, offset: int = 0):
    """The bounded sample of the batch the oracle is timed on: every stride-th graph."""
    return [(g, 0) for g in graphs[offset::stride]]


# ------------------------------------------------------------------ GPU legs

def _events(torch, n):
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]


def batch_leg(args, cc, ctx, graphs, stream, flush, dev, dist):
    """Config 4: the batch resident in HBM, one cc_batch_run + cc_batch_poll per step."""
    import torch
    bs = ctx.load_batch(graphs)
    for _ in range(args.warmup):
        bs.run()
    torch.cuda.synchronize()
    ev = _events(torch, args.steps)
    cyc = paths = 0
    eng_ms = proc_ms = 0.0
    done_all = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            hist, hsh, pth, done, info = bs.run()
            ev[k][1].record(stream)
            cyc += int(hist.sum())
            paths += int(pth.sum())
            eng_ms += info.ms_engine
            proc_ms += info.ms_proc
            done_all.append(done / 1000.0)
        torch.cuda.synchronize()
    t_ms = float(sum(a.elapsed_time(b) for a, b in ev))
    if dist:
        t_ms = max_over_ranks(t_ms, dist, dev)
    world = dist.get_world_size() if dist else 1
    p50, p99 = _percentiles(np.concatenate(done_all))
    K = args.steps
    out = {
        "value": world * cyc / (t_ms / 1000.0), "ms_per_step": t_ms / K, "cycles_per_step": cyc // K,
        "paths_per_step": paths // K, "paths_expanded_per_s": world * paths / (t_ms / 1000.0),
        "per_graph_done_ms": {"p50": p50, "p99": p99, "of": f"{len(graphs)} graphs x {K} steps",
                              "what": "engine start to the end of the step that expanded the graph's last path"},
        "engine_ms_per_step": eng_ms / K, "device_ms_per_step": proc_ms / K,
        "spilled": int(info.spilled), "peak_frontier_bytes": int(info.peak_bytes),
        "gpu_launches": 2 * K,  # labelling + seeding of every graph, one persistent expansion
        "clocks": clk.summary(),
        "roofline": roofline("engine_kernel<Multi,256> (batch expansion)", 2 * bitset_record_bytes(1) * paths / K,
                             eng_ms / K, paths / K, "engine_multi_batch"),
    }
    bs.close()
    return out, hist, hsh


def per_graph_leg(cc, ctx, graphs):
    """The same graphs as 4096 plain cc_enumerate calls (graphs resident; one warm pass so
    that every call replays its captured CUDA graph)."""
    import torch
    loaded = [ctx.load(g) for g in graphs]
    for lg in loaded:
        lg.enumerate()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cyc, dev_ms, launches = 0, 0.0, 0
    for lg in loaded:
        r = lg.enumerate()
        cyc += r.total
        dev_ms += r.info.ms_proc
    wall = time.perf_counter() - t0
    for lg in loaded:
        lg.close()
    return {"value": cyc / wall, "unit": UNIT, "seconds": wall, "device_ms_sum": dev_ms,
            "device_only_value": cyc / (dev_ms / 1000.0) if dev_ms > 0 else None}, cyc


def batch_e2e_leg(cc, ctx, graphs, steps, dist=None, dev=None):
    """End to end through the public API: cc_batch_submit from pinned host buffers (packed
    CSR of every graph: validated, copied to the device) + cc_batch_poll (results copied
    back to the host), wall clock per step."""
    import torch
    packed = I.pack(graphs)
    pinned = []
    for a in packed:
        a = np.ascontiguousarray(a)
        t = torch.from_numpy(a.view(np.int32 if a.dtype == np.uint32 else np.int64)).pin_memory()
        pinned.append(t.numpy().view(a.dtype))
    ns, row_off, rp, col_off, cl = pinned
    h2d = sum(int(a.nbytes) for a in pinned)
    count = len(graphs)
    d2h = 2 * 8 * 65 * count + 8 * count + 4 * count  # histograms, stored-path counts, hashes, finish steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cyc = 0
    for _ in range(steps):
        bid = ctypes_batch_submit(cc, ctx, ns, row_off, rp, col_off, cl)
        while True:
            s, hist, hsh, paths, done, info = cc.cc_batch_poll(ctx.handle, bid, count, 200000)
            if s != cc.CC_PENDING:
                break
        assert s == cc.CC_OK, s
        cyc += int(hist.sum())
    dt = time.perf_counter() - t0
    world = 1
    if dist:
        dt = max_over_ranks(dt, dist, dev)
        world = dist.get_world_size()
    return {"value": world * cyc / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "api": "cc_batch_submit + cc_batch_poll from pinned host buffers"}


def ctypes_batch_submit(cc, ctx, ns, row_off, rp, col_off, cl):
    import ctypes
    bid = ctypes.c_uint64(0)
    u32 = ctypes.POINTER(ctypes.c_uint32)
    u64 = ctypes.POINTER(ctypes.c_uint64)
    s = cc.load_library().cc_batch_submit(ctx.handle, ns.size, ns.ctypes.data_as(u32), row_off.ctypes.data_as(u64),
                                          rp.ctypes.data_as(u32), col_off.ctypes.data_as(u64),
                                          cl.ctypes.data_as(u32), 0, ctypes.byref(bid))
    assert s == cc.CC_OK, s
    return int(bid.value)


def single_leg(args, cc, work, steps, warmup, stream, flush, dev, dist, profile, kernel, span_clocks=False):
    """Single graphs through cc_enumerate on graphs resident in HBM.  With N ranks each rank
    enumerates its share of every graph's initial triplets (cc_enumerate_part) and one
    all-reduce sums the histograms and hashes (strong scaling).  `span_clocks` (the
    sub-objects of the batch line) times enough steps for the clock record; the line of a
    single-graph workload times exactly `steps`."""
    import torch
    rank = dist.get_rank() if dist else 0
    world = dist.get_world_size() if dist else 1
    ctx = cc.Context(frontier_bytes=_frontier_bytes(args, 8 << 10), stream=stream.cuda_stream,
                     flags=cc.CC_FLAG_NO_GRAPH if args.no_graph else 0)
    loaded = [(ctx.load(g), L, g) for g, L in work]

    def step():
        res = [lg.enumerate(L, part=rank, nparts=world) for lg, L, _ in loaded]
        # the exchange step of a split graph: one all-reduce of its histogram and hash
        return res, [sum_results(r.hist, r.hash, dist, dev) for r in res] if dist else None

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if span_clocks:
        # a step takes about a millisecond: time enough of them for the clock record
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        steps = steps_for_clocks(steps, (time.perf_counter() - t0) * 1000.0, dist, dev)
    ev = _events(torch, steps)
    cycles = paths = 0
    eng_ms, alg, launches = 0.0, 0, 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clk:
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            res, summed = step()
            ev[k][1].record(stream)
            for (lg, L, g), r in zip(loaded, res):
                cycles += r.total
                paths += r.paths
                eng_ms += r.info.ms_engine
                alg += algorithmic_bytes(r.tcount, g.n, int(r.info.mode))
                launches += int(r.info.launches)
        torch.cuda.synchronize()
    t_ms = float(sum(a.elapsed_time(b) for a, b in ev))
    local_paths = paths
    if dist:
        t_ms = max_over_ranks(t_ms, dist, dev)
        # paths were expanded by the rank that owns their triplet: summed over ranks; the
        # cycles of each step were summed by the step's own exchange
        tot = torch.tensor([paths], dtype=torch.int64, device=dev)
        dist.all_reduce(tot)
        paths = int(tot[0])
        cycles = steps * sum(int(h.sum()) for h, _ in summed)
    # end to end through the public API: H2D of the CSR from pinned memory (cc_graph_load),
    # enumeration, D2H of the results, free
    pinned = []
    for g, L in work:
        rp = torch.from_numpy(g.row_ptr.astype(np.uint32).view(np.int32)).pin_memory()
        cl = torch.from_numpy(g.col.astype(np.uint32).view(np.int32)).pin_memory()
        pinned.append((g, L, rp.numpy().view(np.uint32), cl.numpy().view(np.uint32)))
    h2d = sum(4 * (rp.size + cl.size) for _, _, rp, cl in pinned)
    d2h = sum(8 * (2 * ((L or g.n) + 1) + 1) for g, L, _, _ in pinned)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(steps, 10))
    t0 = time.perf_counter()
    ecyc = 0
    for _ in range(e2e_steps):
        for g, L, rp, cl in pinned:
            s, h = cc.cc_graph_load(ctx.handle, g.n, rp, cl)
            assert s == cc.CC_OK
            s, hist, hh, tc, _, info = cc.cc_enumerate(h, g.n, L, part=rank, nparts=world)
            assert s == cc.CC_OK
            ecyc += int(hist.sum())
            cc.cc_graph_free(h)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:
        e2e_s = max_over_ranks(e2e_s, dist, dev)
        t = torch.tensor([ecyc], dtype=torch.int64, device=dev)
        dist.all_reduce(t)
        ecyc = int(t[0])
    for lg, _, _ in loaded:
        lg.close()
    ctx.close()
    return {
        "value": cycles / (t_ms / 1000.0), "unit": UNIT, "ms_per_step": t_ms / steps, "steps": steps,
        "cycles_per_step": cycles // steps, "paths_per_step": paths // steps,
        "paths_expanded_per_s": paths / (t_ms / 1000.0),
        "roofline": roofline(kernel, alg / steps, eng_ms / steps, local_paths / steps, profile),
        "e2e": {"value": ecyc / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "api": "cc_graph_load + cc_enumerate + cc_graph_free from pinned host CSR"},
        "gpu_launches": launches, "clocks": clk.summary(),
    }


def serve_leg(args):
    """Config 5: Poisson arrivals (seed 3) of serving requests, continuous batching,
    latency p50/p99 from arrival to result, against sequential per-graph launches."""
    import torch

    from paper_1410_4876_gb300 import cc
    arrivals = I.poisson_arrivals(args.rate, args.serve_seconds, 3)
    reqs = [I.make(*I.serving_request(i, 3)) for i in range(len(arrivals))]
    n_req = len(reqs)
    ctx = cc.Context(frontier_bytes=_frontier_bytes(args, 64 << 10))
    srv = cc.Server(ctx, slots=4096, steps_per_round=args.serve_steps, admit_bytes=64 << 30)
    for g in reqs[:8]:  # warm up the kernels on a few requests
        srv.submit(g)
    left = 8
    while left:
        d, _, _ = srv.step()
        left -= len(d)
    torch.cuda.synchronize()
    ids, lat, waits = {}, [], []
    cyc = paths = 0
    i = finished = rounds = 0
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        while finished < n_req:
            now = time.perf_counter() - t0
            while i < n_req and arrivals[i] <= now:
                ids[srv.submit(reqs[i])] = i
                i += 1
            done, inflight, queued = srv.step()
            rounds += 1
            tnow = time.perf_counter() - t0
            for d in done:
                k = ids.pop(d["id"])
                lat.append(tnow - arrivals[k])
                waits.append(d["wait_us"] / 1e6)
                cyc += d["total"]
                paths += d["paths"]
            finished += len(done)
            if inflight == 0 and queued == 0 and i < n_req:
                while time.perf_counter() - t0 < arrivals[i]:
                    pass
        elapsed = time.perf_counter() - t0
    srv.close()
    p50, p99 = _percentiles(np.array(lat) * 1000)
    w50, w99 = _percentiles(np.array(waits) * 1000)
    # plain sequential per-graph launches on a prefix of the same stream
    k = min(n_req, args.seq_sample)
    t1 = time.perf_counter()
    seq_c = 0
    for g in reqs[:k]:
        seq_c += ctx.enumerate(g).total
    t_seq = time.perf_counter() - t1
    ctx.close()
    return {
        "metric": "served chordless cycles/s", "value": cyc / elapsed, "unit": UNIT,
        "workload": f"Poisson arrivals, mean {args.rate:g}/s for {args.serve_seconds:g} s (seed 3): 95% batch-mixture "
                    "graphs + 5% 8x8 grids; admission budget 64 GiB of predicted frontier",
        "requests": n_req, "rounds": rounds, "steps_per_round": args.serve_steps,
        "offered_requests_per_s": n_req / args.serve_seconds, "achieved_requests_per_s": n_req / elapsed,
        "elapsed_s": elapsed, "paths_expanded_per_s": paths / elapsed,
        "latency_ms": {"p50": p50, "p99": p99, "what": "arrival to result on the host"},
        "queue_wait_ms": {"p50": w50, "p99": w99},
        "sequential_per_graph": {"requests": k, "requests_per_s": k / t_seq, "cycles_per_s": seq_c / t_seq},
        "clocks": clk.summary(),
    }


def stream_leg(args):
    """Every cycle of Table 1's 8 x 10 grid (71.5 M, counted without being stored in the
    paper) listed through cc_enumerate_stream: device lists of --stream-chunk cycles, each
    round's lists copied to pinned host memory and handed to a sink that checks them
    (cycle count and length histogram).  Wall time of the whole call, sink included."""
    import torch

    from paper_1410_4876_gb300 import cc
    g = I.grid(8, 10)
    chunk_c = args.stream_chunk
    chunk_v = 24 * chunk_c
    ctx = cc.Context(frontier_bytes=_frontier_bytes(args, 32 << 10))
    lg = ctx.load(g)
    ref = lg.enumerate()
    acc = {"cycles": 0, "verts": 0}

    def sink(starts, lengths, verts):
        acc["cycles"] += len(lengths)
        acc["verts"] += int(lengths.sum(dtype=np.int64))

    for _ in range(args.warmup):
        lg.enumerate_stream(sink, 0, chunk_c, chunk_v)
    torch.cuda.synchronize()
    times = []
    rounds = 0
    for _ in range(args.steps):
        acc["cycles"] = acc["verts"] = 0
        t0 = time.perf_counter()
        r, rounds = lg.enumerate_stream(sink, 0, chunk_c, chunk_v)
        times.append(time.perf_counter() - t0)
        assert acc["cycles"] == r.total == ref.total and r.hash == ref.hash
        assert acc["verts"] == sum(k * int(c) for k, c in enumerate(r.hist))
    t = min(times)
    t_count = ref.info.ms_total / 1000.0
    out_bytes = 12 * acc["cycles"] + 4 * acc["verts"]
    line = {
        "metric": "streamed chordless cycles/s", "value": acc["cycles"] / t, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "grid 8x10 (80 vertices, 142 edges), every chordless cycle listed "
                               "(Table 1's count-only row)", "cycles": acc["cycles"], "vertices": acc["verts"],
                   "chunk_cycles": chunk_c, "chunk_vertices": chunk_v},
        "rounds": rounds, "steps_expansion": int(r.info.steps), "engine_ms": r.info.ms_engine,
        "host_bytes_per_s": out_bytes / t, "bytes_to_host": out_bytes,
        "count_only": {"value": ref.total / t_count, "unit": UNIT, "ms": 1000 * t_count},
    }
    lg.close()
    ctx.close()
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ the two arms

def _base_line(args, world, value, ms, desc, extra_config=None):
    cfg = {"workload": desc, "l2": "flushed before every timed step (256 MiB write)",
           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}
    cfg.update(extra_config or {})
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg}


def run_ours_batch(args):
    import torch

    from paper_1410_4876_gb300 import cc
    rank, world, local = _env_rank()
    dist = _dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    graphs = I.mixture(args.batch_count, 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # twice the 129 MB L2
    ctx = cc.Context(frontier_bytes=_frontier_bytes(args, 64 << 10), stream=stream.cuda_stream)
    out, hist, hsh = batch_leg(args, cc, ctx, graphs, stream, flush, dev, dist)
    pg, seq_cyc = per_graph_leg(cc, ctx, graphs)
    assert seq_cyc == out["cycles_per_step"], (seq_cyc, out["cycles_per_step"])
    e2e = batch_e2e_leg(cc, ctx, graphs, max(1, min(args.steps, 5)), dist, dev)
    ctx.close()
    line = _base_line(args, world, out["value"], out["ms_per_step"], batch_desc(len(graphs)),
                      {"graphs": len(graphs), "cycles_per_step": out["cycles_per_step"],
                       "paths_per_step": out["paths_per_step"], "seed": 0})
    line["paths_expanded_per_s"] = out["paths_expanded_per_s"]
    line["batched_over_per_graph"] = out["value"] / world / pg["value"]
    line["per_graph_launches"] = pg
    line["per_graph_done_ms"] = out["per_graph_done_ms"]
    line["roofline"] = out["roofline"]
    line["e2e"] = e2e
    line["gpu_launches"] = out["gpu_launches"]
    line["clocks"] = out["clocks"]
    for k in ("engine_ms_per_step", "device_ms_per_step", "spilled", "peak_frontier_bytes"):
        line[k] = out[k]
    if rank == 0 and not args.no_cpu:
        stride = args.cpu_stride
        line["cpu_baseline"] = cpu_baseline_line(batch_sample(graphs, stride),
                                                 f"every {stride}th graph of the batch ({len(graphs[::stride])} graphs)")
    if world == 1 and not args.no_sub:
        subs = {}
        for key, profile, kernel in (("grid8+gnp60", "engine_bitset1_grid8_gnp60", "engine_kernel<Bitset1,256>"),
                                     ("gnm2000", "engine_csr16_gnm2000_len12", "engine_kernel<Csr16,256>")):
            desc, make = WORKLOADS[key]
            work = make()
            sub = single_leg(args, cc, work, min(args.steps, 10), args.warmup, stream, flush, dev, None, profile,
                             kernel, span_clocks=True)
            sub["workload"] = desc
            if not args.no_cpu:
                sub["cpu_baseline"] = cpu_baseline_line(work, "whole workload")
            subs[key] = sub
        line["single_graph"] = subs
        if not args.no_serve:
            line["serving"] = serve_leg(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_ours_single(args, work, desc, profile, kernel):
    import torch

    from paper_1410_4876_gb300 import cc
    rank, world, local = _env_rank()
    dist = _dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sub = single_leg(args, cc, work, args.steps, args.warmup, stream, flush, dev, dist, profile, kernel)
    line = _base_line(args, world, sub["value"], sub["ms_per_step"], desc,
                      {"cycles_per_step": sub["cycles_per_step"], "paths_per_step": sub["paths_per_step"]})
    if world > 1:
        line["scaling"] = "strong"
        line["config"]["parallelism"] = f"initial triplets split over {world} ranks, one all-reduce of the results"
    for k in ("paths_expanded_per_s", "roofline", "e2e", "gpu_launches", "clocks"):
        line[k] = sub[k]
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_line(work, "whole workload")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_reference(args):
    """The oracle as it stands on the host cores, same workload and metric; each step a
    bounded sample: a rotating 1/512 of the batch's graphs, or a rotating quarter of a single
    graph's initial-triplet parts.  Rank 0 only."""
    import oracle
    import concurrent.futures as cf
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    if args.workload == "batch":
        graphs = I.mixture(args.batch_count, 0)
        R = 512
        desc = batch_desc(len(graphs))
        sample = f"each step: every {R}th graph of the batch from a rotating offset, triplets split on {cores} threads"

        def one(s):
            c, p, dt, _ = cpu_oracle(batch_sample(graphs, R, s % R))
            return c, p, dt
    else:
        desc, make = WORKLOADS[args.workload]
        work = make()
        nparts = cores * 4
        sample = f"each step: every 4th of {nparts} initial-triplet parts (rotating), {cores} threads"

        def one(s):
            parts = list(range(s % 4, nparts, 4))
            t0 = time.perf_counter()
            with cf.ThreadPoolExecutor(cores) as ex:
                res = list(ex.map(lambda j: oracle.enumerate_cycles(j[0], max_len=j[1], part=j[2], nparts=nparts),
                                  [(g, L, p) for g, L in work for p in parts]))
            return sum(r.total for r in res), sum(int(r.tcount.sum()) for r in res), time.perf_counter() - t0

    for w in range(args.warmup):
        one(10_000 + w)
    tot_c = tot_p = 0
    tot_t = 0.0
    for s in range(args.steps):
        c, p, dt = one(s)
        tot_c += c
        tot_p += p
        tot_t += dt
    value = tot_c / tot_t if tot_t > 0 else 0.0
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": desc, "sample": sample},
        "paths_expanded_per_s": tot_p / tot_t if tot_t > 0 else 0.0,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch", choices=["batch"] + sorted(WORKLOADS) + ["serve", "stream"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline legs")
    ap.add_argument("--no-sub", action="store_true", help="batch: skip the single-graph and serving sub-objects")
    ap.add_argument("--no-serve", action="store_true", help="batch: skip the serving sub-object")
    ap.add_argument("--frontier-mb", type=int, default=0,
                    help="device memory for paths in flight (MiB); 0 = 8 GiB for single graphs, "
                         "64 GiB for the batch and serving workloads (whose frontiers hold many graphs)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel directly (no CUDA-graph replay of repeated enumerations)")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--cpu-stride", type=int, default=16, help="batch: the oracle is timed on every n-th graph")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: mean arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serving: arrival window (s)")
    ap.add_argument("--serve-steps", type=int, default=8, help="serving: expansion steps per round")
    ap.add_argument("--seq-sample", type=int, default=2000, help="serving: requests timed one by one")
    ap.add_argument("--stream-chunk", type=int, default=32 << 20, help="stream: device list capacity (cycles)")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.workload in ("serve", "stream"):
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the batch and the "
                              "single-graph workloads"}))
            return
        return run_reference(args)
    if args.workload == "batch":
        return run_ours_batch(args)
    if args.workload == "serve":
        line = serve_leg(args)
        line.update({"n_gpus": 1, "steps": line["rounds"], "warmup": 1, "higher_is_better": True,
                     "ms_per_step": 1000 * line["elapsed_s"] / max(line["rounds"], 1), "scaling": "weak",
                     "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                     "config": {"workload": line.pop("workload")}})
        print(json.dumps(line), flush=True)
        return
    if args.workload == "stream":
        return stream_leg(args)
    desc, make = WORKLOADS[args.workload]
    profile, kernel = {"gnm2000": ("engine_csr16_gnm2000_len12", "engine_kernel<Csr16,256>")}.get(
        args.workload, ("engine_bitset1_grid8_gnp60", "engine_kernel<Bitset1,256>"))
    run_ours_single(args, make(), desc, profile, kernel)


if __name__ == "__main__":
    main()
