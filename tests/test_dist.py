"""The multi-rank path of bench.py on CPU with two gloo ranks: the timing reduced to the
slowest rank, and the exchange step of a graph split over its initial triplets (each rank
enumerates its part with the oracle; one all-reduce of histogram and hash gives the whole
graph's result)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    out[rank] = t
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 15.0, 1: 15.0}


def _part_worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_1410_4876_gb300 import inputs as I
    res = {}
    for name, g in (("grid8", I.grid(8, 8)), ("gnp60", I.gnp(60, 0.15, 7))):
        r = oracle.enumerate_cycles(g, part=rank, nparts=world)
        h, hh = bench.sum_results(r.hist, r.hash, dist)
        res[name] = (h.tolist(), hh, r.total)
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_split_triplets_sum_to_the_whole():
    import oracle
    from paper_1410_4876_gb300 import inputs as I
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_part_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for name, g in (("grid8", I.grid(8, 8)), ("gnp60", I.gnp(60, 0.15, 7))):
        whole = oracle.enumerate_cycles(g)
        for rank in range(2):
            h, hh, part_total = out[rank][name]
            assert h == whole.hist.tolist() and hh == whole.hash
            assert 0 < part_total < whole.total  # each rank did a real share


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
