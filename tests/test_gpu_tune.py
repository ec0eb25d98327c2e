"""Launch variants give identical results: CUDA-graph replay against direct launches, the
runtime knobs (paths per thread, cluster-phase size, launch shape), and the autotuner, which
times those variants and must find them all in agreement.  Bit-exact against the oracle
where the graph is small enough."""
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


def _same(r, ref):
    assert r.hist.tolist() == ref.hist.tolist()
    assert r.hash == ref.hash
    assert r.tcount.tolist() == ref.tcount.tolist()


# every case finishes in the oracle within a second (sparse random graphs with all cycle
# lengths are kept to mean degree <= 2.4 on <= 200 vertices: denser or larger ones have
# astronomically many chordless cycles)
GRAPHS = [I.grid(6, 6), I.gnp(40, 0.12, 3), I.gnp(100, 2.4 / 100, 100), I.gnp(200, 1.9 / 200, 200)]
_REF = {}


def _ref(g, L=0):
    key = (g.name, L)
    if key not in _REF:
        _REF[key] = oracle.enumerate_cycles(g, max_len=L)
    return _REF[key]


@pytest.mark.parametrize("g,L", [(g, 0) for g in GRAPHS] + [(I.gnm(400, 800, 9), 10)],
                         ids=lambda x: x.name if hasattr(x, "name") else str(x))
def test_graph_replay_equals_direct(cc, g, L):
    ref = _ref(g, L)
    with cc.Context(frontier_bytes=1 << 30) as ctx, ctx.load(g) as lg:
        runs = [lg.enumerate(L) for _ in range(4)]
    assert [r.info.replayed for r in runs] == [0, 1, 1, 1]
    for r in runs:
        _same(r, ref)
        assert r.info.launches in (3, 4)
        # the replayed graph records the timing events too
        assert 0 < r.info.ms_engine <= r.info.ms_proc <= r.info.ms_total
    # and leaves no CUDA error behind for the caller's next call
    import torch
    assert torch.ones(8, device="cuda").sum().item() == 8
    with cc.Context(frontier_bytes=1 << 30, flags=cc.CC_FLAG_NO_GRAPH) as ctx, ctx.load(g) as lg:
        runs = [lg.enumerate(L) for _ in range(3)]
    assert [r.info.replayed for r in runs] == [0, 0, 0]
    for r in runs:
        _same(r, ref)


def test_replay_follows_length_and_options(cc):
    g = I.grid(5, 6)
    with cc.Context(frontier_bytes=1 << 30) as ctx, ctx.load(g) as lg:
        for L in [0, 8, 0, 8, 12, 12, 0]:
            _same(lg.enumerate(L), _ref(g, L))
        o = cc.cc_options()
        o.paths_per_thread = 1
        ctx.set_options(o)
        for _ in range(3):
            _same(lg.enumerate(), _ref(g))


@pytest.mark.parametrize("pf", [1, 2, 3, 4])
@pytest.mark.parametrize("small", [0, 1024, 1 << 20])
def test_paths_per_thread_and_small_phase(cc, pf, small):
    with cc.Context(frontier_bytes=1 << 30, paths_per_thread=pf, small_phase_paths=small) as ctx:
        for g in GRAPHS:
            _same(ctx.enumerate(g), _ref(g))


@pytest.mark.parametrize("tpb,bps", [(64, 1), (128, 2), (192, 3), (256, 4)])
def test_launch_shapes(cc, tpb, bps):
    with cc.Context(frontier_bytes=1 << 30, threads_per_block=tpb, blocks_per_sm=bps) as ctx:
        for g in [GRAPHS[0], GRAPHS[2]]:
            _same(ctx.enumerate(g), _ref(g))
        g = I.gnm(400, 800, 9)
        _same(ctx.enumerate(g, max_len=10), _ref(g, 10))


def test_set_options_validation(cc):
    with cc.Context(frontier_bytes=1 << 26) as ctx:
        o = cc.cc_options()
        o.paths_per_thread = 5
        assert cc.cc_context_set_options(ctx.handle, o) == cc.CC_ERR_ARG
        o.paths_per_thread = 0
        o.threads_per_block = 96 + 1
        assert cc.cc_context_set_options(ctx.handle, o) == cc.CC_ERR_ARG
        o.threads_per_block = 128
        assert cc.cc_context_set_options(ctx.handle, o) == cc.CC_OK


@pytest.mark.parametrize("g,L", [(I.grid(6, 6), 0), (I.gnp(60, 0.12, 8), 0), (I.gnm(400, 800, 9), 10)],
                         ids=["grid6x6", "gnp60", "gnm400"])
def test_tune_single_and_cache(cc, tmp_path, g, L):
    cache = str(tmp_path / "tune.jsonl")
    ref = _ref(g, L)
    with cc.Context(frontier_bytes=1 << 30) as ctx, ctx.load(g) as lg:
        t = lg.tune(L, cache)
        assert t.from_cache == 0 and t.candidates >= 9
        assert t.ms_best <= t.ms_default
        cls = t.graph_class.decode()
        assert cls.startswith("single:")
        t2 = lg.tune(L, cache)
        assert t2.from_cache == 1 and t2.candidates == 0 and t2.graph_class.decode() == cls
        for f in ["threads_per_block", "blocks_per_sm", "paths_per_thread", "small_phase_paths", "mode", "flags"]:
            assert getattr(t2.best, f) == getattr(t.best, f)
        ctx.set_options(t.best)
        _same(lg.enumerate(L), ref)
        _same(lg.enumerate(L), ref)
    lines = open(cache).read().strip().split("\n")
    assert len(lines) == 1 and '"class": "%s"' % cls in lines[0]


def test_tune_batch(cc, tmp_path):
    graphs = I.mixture(48, 21)
    cache = str(tmp_path / "tune.jsonl")
    with cc.Context(frontier_bytes=2 << 30) as ctx:
        hist0, hash0, _, _, _ = ctx.batch(graphs, max_len=8)
        t = ctx.tune_batch(graphs, 8, cache)
        assert t.from_cache == 0 and t.candidates >= 9
        assert t.graph_class.decode().startswith("batch:")
        ctx.set_options(t.best)
        hist1, hash1, _, _, _ = ctx.batch(graphs, max_len=8)
        assert np.array_equal(hist0, hist1) and np.array_equal(hash0, hash1)
        assert ctx.tune_batch(graphs, 8, cache).from_cache == 1
    for k in range(0, 48, 7):
        ref = oracle.enumerate_cycles(graphs[k], max_len=8)
        assert int(hash1[k]) == ref.hash and hist1[k][: len(ref.hist)].tolist() == ref.hist.tolist()
