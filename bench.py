"""Benchmark: chordless cycles/s (and paths expanded/s) on one GB300.

Default workload (one step): full enumeration of the 8 x 8 grid graph and of the seeded
Erdos-Renyi graph G(n=60, p=0.15, seed 7), all cycle lengths, through the C ABI
(cc_enumerate on graphs already resident in HBM).  Between timed steps the L2 cache is
flushed by writing a 256 MiB buffer (about twice the L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload grid8+gnp60|grid6|grid7x10|grid8x10|gnm2000|batch|serve|stream]

--impl reference times the CPU oracle (Algorithm 1 in plain C, test infrastructure) on
the host cores for the same workload and metric.  Under torchrun (N > 1) every rank runs
its own replica of the workload (independent problems, no collective): weak scaling.
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1410_4876_gb300 import inputs as I  # noqa: E402

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


def unstored_levels(tcount, expanded) -> set:
    """Levels that two-level steps expanded without storing them, from the per-step trace
    (a step expands one level, or a level and its children; chunked steps of a spilled run
    are not resolved and count every level as stored)."""
    nz = [t for t in range(len(tcount)) if tcount[t]]
    skip, i = set(), 0
    for e in (int(x) for x in expanded):
        if i < len(nz) and e == int(tcount[nz[i]]):
            i += 1
        elif i + 1 < len(nz) and e == int(tcount[nz[i]]) + int(tcount[nz[i + 1]]):
            skip.add(nz[i + 1])
            i += 2
        else:
            return set()
    return skip if i == len(nz) else set()


def algorithmic_bytes(r, n: int, skip=()) -> int:
    """Bytes the expansion kernel must move: every stored path is read once and every
    stored path after the initial triplets is written once (levels in `skip` were expanded
    inside a two-level step and never stored).  Record sizes: bitset, n <= 64:
    B (8) + H (8) + M (4) = 20 bytes; n <= 128: 28; n <= 256: 44; CSR: the path's u16 ids
    padded to a multiple of 8 (16 bytes for t <= 8, 32 for t <= 16, ...)."""
    tc = r.tcount.astype(np.int64).copy()
    if tc.size <= 3:
        return 0
    for t in skip:
        tc[t] = 0
    if r.info.mode == 2:
        t = np.arange(tc.size, dtype=np.int64)
        rec = (t + 7) // 8 * 16
        return int((tc * rec).sum() * 2 - int(tc[3]) * 16)
    rec = 20 if n <= 64 else (28 if n <= 128 else 44)
    return rec * (2 * int(tc.sum()) - int(tc[3]))


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
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_baseline(work, seconds_hint=True, parts_per_core=2, sample_parts=None):
    """The oracle as it stands, run over the workload's initial triplets split across all
    host cores (threads; ctypes releases the GIL).  ``sample_parts`` limits the run to a
    subset of the parts (a bounded sample)."""
    import concurrent.futures as cf

    import oracle
    cores = os.cpu_count() or 1
    nparts = cores * parts_per_core
    parts = list(range(nparts)) if sample_parts is None else sample_parts
    t0 = time.perf_counter()
    cyc = paths = 0
    with cf.ThreadPoolExecutor(cores) as ex:
        for g, L in work:
            res = list(ex.map(lambda p: oracle.enumerate_cycles(g, max_len=L, part=p, nparts=nparts), parts))
            cyc += sum(r.total for r in res)
            paths += sum(int(r.tcount.sum()) for r in res)
    dt = time.perf_counter() - t0
    return cyc, paths, dt, cores, len(parts), nparts


def run_reference(args, work, desc):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    nparts = cores * 4
    # each step: a quarter of the triplet parts (rotating), one part per host core
    for w in range(args.warmup):
        cpu_baseline(work, parts_per_core=4, sample_parts=list(range(w % 4, nparts, 4)))
    tot_c = tot_p = 0
    tot_t = 0.0
    for s in range(args.steps):
        c, p, dt, _, _, _ = cpu_baseline(work, parts_per_core=4, sample_parts=list(range(s % 4, nparts, 4)))
        tot_c += c
        tot_p += p
        tot_t += dt
    value = tot_c / tot_t if tot_t > 0 else 0.0
    line = {
        "impl": "reference", "metric": "chordless cycles/s", "value": value, "unit": "cycles/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": desc, "sample": "each step: every 4th of the initial-triplet parts (rotating)"},
        "paths_expanded_per_s": tot_p / tot_t if tot_t > 0 else 0.0,
        "cpu_baseline": {"value": value, "unit": "cycles/s", "cores": cores, "kind": "oracle",
                         "sample": f"{nparts} triplet parts, a quarter per step, {cores} threads"},
        "e2e": {"value": value, "unit": "cycles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, work, desc):
    import torch

    from paper_1410_4876_gb300 import cc
    rank, world, local = _env_rank()
    dist = _dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    # run on torch's stream so events, the L2 flush and the library share one stream
    ctx = cc.Context(frontier_bytes=_frontier_bytes(args, 8 << 10), stream=stream.cuda_stream,
                     flags=cc.CC_FLAG_NO_GRAPH if args.no_graph else 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # twice the 129 MB L2
    loaded = [(ctx.load(g), L, g) for g, L in work]

    def step():
        res = [lg.enumerate(L) for lg, L, _ in loaded]
        return res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    cycles = paths = 0
    eng_ms = 0.0
    eng_bytes = 0
    launches = 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            res = step()
            ev[k][1].record(stream)
            for r in res:
                cycles += r.total
                paths += r.paths
                eng_ms += r.info.ms_engine
                launches += int(r.info.launches)
        torch.cuda.synchronize()
    # algorithmic bytes per step: the stored levels of each graph, from one more call's trace
    for lg, L, g in loaded:
        r = lg.enumerate(L)
        _, expanded = cc.cc_get_trace(ctx.handle)
        eng_bytes += args.steps * algorithmic_bytes(r, g.n, unstored_levels(r.tcount, expanded))
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = float(sum(step_ms))
    if dist:
        t_ms = max_over_ranks(t_ms, dist, dev)
        dist.barrier()
    value = world * cycles / (t_ms / 1000.0)

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
    e2e_steps = max(1, min(args.steps, 10))
    t0 = time.perf_counter()
    ecyc = 0
    for _ in range(e2e_steps):
        for g, L, rp, cl in pinned:
            s, h = cc.cc_graph_load(ctx.handle, g.n, rp, cl)
            assert s == cc.CC_OK
            s, hist, hh, tc, _, info = cc.cc_enumerate(h, g.n, L)
            assert s == cc.CC_OK
            ecyc += int(hist.sum())
            cc.cc_graph_free(h)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * ecyc / e2e_s

    peak, peak_kind = _peaks()
    achieved = eng_bytes / (eng_ms / 1000.0) / 1e9 if eng_ms > 0 else 0.0
    traffic = _ncu_traffic(args.workload)
    line = {
        "metric": "chordless cycles/s", "value": value, "unit": "cycles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": desc, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "cycles_per_step": cycles // args.steps, "paths_per_step": paths // args.steps},
        "paths_expanded_per_s": world * paths / (t_ms / 1000.0),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if peak else None, "traffic": traffic,
                     "kernel": "engine_kernel (persistent expansion)", "peak_kind": peak_kind,
                     "algorithmic_bytes_per_step": eng_bytes // args.steps, "kernel_ms_per_step": eng_ms / args.steps},
        "e2e": {"value": e2e_value, "unit": "cycles/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu:
        c, p, dt, cores, nsel, nparts = cpu_baseline(work, sample_parts=None)
        line["cpu_baseline"] = {"value": c / dt, "unit": "cycles/s", "cores": cores, "kind": "oracle",
                                "sample": f"whole workload, {nparts} triplet parts on {cores} threads, {dt:.1f} s"}
    for lg, _, _ in loaded:
        lg.close()
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _percentiles(x):
    x = np.asarray(x, dtype=np.float64)
    if x.size == 0:
        return None, None
    return float(np.percentile(x, 50)), float(np.percentile(x, 99))


def _frontier_bytes(args, default_mb):
    return (args.frontier_mb or default_mb) << 20


def run_batch(args):
    """4096 graphs of the batch mixture (seed 0) in one persistent launch, against plain
    per-graph cc_enumerate calls of the same graphs."""
    import torch

    from paper_1410_4876_gb300 import cc
    graphs = I.mixture(args.batch_count, 0)
    ctx = cc.Context(frontier_bytes=_frontier_bytes(args, 64 << 10))
    for _ in range(args.warmup):
        ctx.batch(graphs[:256])
    torch.cuda.synchronize()
    times, cyc, paths, p50, p99 = [], 0, 0, None, None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        hist, hsh, pth, done, info = ctx.batch(graphs)
        times.append(time.perf_counter() - t0)
        cyc, paths = int(hist.sum()), int(pth.sum())
        p50, p99 = _percentiles(done / 1000.0)
        eng_ms = info.ms_engine
        last_info = info
    t = min(times)
    # plain per-graph launches (label + seed + expansion kernels per graph), same graphs
    loaded = [ctx.load(g) for g in graphs]
    t0 = time.perf_counter()
    seq_cyc = 0
    for lg in loaded:
        seq_cyc += lg.enumerate().total
    t_seq = time.perf_counter() - t0
    for lg in loaded:
        lg.close()
    assert seq_cyc == cyc
    line = {
        "metric": "chordless cycles/s (batched)", "value": cyc / t, "unit": "cycles/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{len(graphs)} graphs of the seeded batch mixture (50% G(n,p), 30% grids, "
                               "20% K_ab), all lengths", "cycles": cyc, "paths": paths},
        "paths_expanded_per_s": paths / t, "engine_ms": eng_ms, "spilled": int(last_info.spilled),
        "peak_frontier_bytes": int(last_info.peak_bytes), "frontier_bytes": _frontier_bytes(args, 64 << 10),
        "per_graph_done_ms": {"p50": p50, "p99": p99},
        "per_graph_launches": {"value": seq_cyc / t_seq, "unit": "cycles/s", "seconds": t_seq},
        "batched_over_per_graph": (cyc / t) / (seq_cyc / t_seq),
    }
    ctx.close()
    print(json.dumps(line), flush=True)


def run_stream(args):
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
        "metric": "streamed chordless cycles/s", "value": acc["cycles"] / t, "unit": "cycles/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "grid 8x10 (80 vertices, 142 edges), every chordless cycle listed "
                               "(Table 1's count-only row)", "cycles": acc["cycles"], "vertices": acc["verts"],
                   "chunk_cycles": chunk_c, "chunk_vertices": chunk_v},
        "rounds": rounds, "steps_expansion": int(r.info.steps), "engine_ms": r.info.ms_engine,
        "host_bytes_per_s": out_bytes / t, "bytes_to_host": out_bytes,
        "count_only": {"value": ref.total / t_count, "unit": "cycles/s", "ms": 1000 * t_count},
    }
    lg.close()
    ctx.close()
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Poisson arrivals (seed 3) of serving requests, continuous batching, p50/p99."""
    import torch

    from paper_1410_4876_gb300 import cc
    arrivals = I.poisson_arrivals(args.rate, args.serve_seconds, 3)
    reqs = [I.make(*I.serving_request(i, 3)) for i in range(len(arrivals))]
    n_req = len(reqs)
    ctx = cc.Context(frontier_bytes=_frontier_bytes(args, 64 << 10))
    srv = cc.Server(ctx, slots=4096, steps_per_round=args.serve_steps, admit_bytes=64 << 30)
    # warm up the kernels on a few requests
    for g in reqs[:8]:
        srv.submit(g)
    left = 8
    while left:
        d, _, _ = srv.step()
        left -= len(d)
    torch.cuda.synchronize()
    ids, lat, waits = {}, [], []
    cyc = paths = 0
    i = 0
    finished = 0
    rounds = 0
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
    line = {
        "metric": "served chordless cycles/s", "value": cyc / elapsed, "unit": "cycles/s", "n_gpus": 1,
        "steps": rounds, "warmup": 1, "ms_per_step": 1000 * elapsed / max(rounds, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"Poisson arrivals, mean {args.rate}/s for {args.serve_seconds} s (seed 3): "
                               "95% batch-mixture graphs + 5% 8x8 grids; admission budget 64 GiB",
                   "requests": n_req, "steps_per_round": args.serve_steps},
        "offered_requests_per_s": n_req / args.serve_seconds, "achieved_requests_per_s": n_req / elapsed,
        "elapsed_s": elapsed, "paths_expanded_per_s": paths / elapsed,
        "latency_ms": {"p50": p50, "p99": p99}, "queue_wait_ms": {"p50": w50, "p99": w99},
        "sequential_per_graph": {"requests": k, "requests_per_s": k / t_seq, "cycles_per_s": seq_c / t_seq},
    }
    print(json.dumps(line), flush=True)


def _engine_fingerprint() -> str:
    """Hash of the engine's code (cc_engine.cu + cc_internal.cuh without comments and
    whitespace), so that a committed ncu capture is used only for the code it measured."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1410_4876_gb300", "csrc")
    text = ""
    for f in ("cc_engine.cu", "cc_internal.cuh"):
        src = open(os.path.join(csrc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        text += re.sub(r"\s+", "", src)
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def _ncu_traffic(workload: str):
    """DRAM bytes per step of the expansion kernel from the committed ncu summary, only
    when that summary was captured on this workload and on the current engine source
    (its fingerprint matches); otherwise None."""
    if workload != "grid8+gnp60":
        return None
    p = os.path.join(ROOT, "profiles", "engine_bitset1_grid8_gnp60.json")
    try:
        d = json.load(open(p))
        if d.get("source_fingerprint") != _engine_fingerprint():
            return None
        return d.get("dram_bytes_per_step")
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid8+gnp60", choices=sorted(WORKLOADS) + ["batch", "serve", "stream"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--frontier-mb", type=int, default=0,
                    help="device memory for paths in flight (MiB); 0 = 8 GiB for single graphs, "
                         "64 GiB for the batch and serving workloads (whose frontiers hold many graphs)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel directly (no CUDA-graph replay of repeated enumerations)")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: mean arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serving: arrival window (s)")
    ap.add_argument("--serve-steps", type=int, default=8, help="serving: expansion steps per round")
    ap.add_argument("--seq-sample", type=int, default=2000, help="serving: requests timed one by one")
    ap.add_argument("--stream-chunk", type=int, default=32 << 20, help="stream: device list capacity (cycles)")
    args = ap.parse_args()
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "stream":
        return run_stream(args)
    desc, make = WORKLOADS[args.workload]
    work = make()
    if args.impl == "reference":
        run_reference(args, work, desc)
    else:
        run_ours(args, work, desc)


if __name__ == "__main__":
    main()
