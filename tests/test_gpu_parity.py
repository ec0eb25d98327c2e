"""CUDA path against the CPU oracle, element by element, through the C ABI.

Integer results, so the bar is bit-exact: per-length histogram, total, 64-bit cycle hash,
per-length stored-path counts (same degree labelling and tie rule on both sides) and,
where requested, the canonical cycle lists.
"""
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


@pytest.fixture(scope="module")
def ctx(cc):
    c = cc.Context(frontier_bytes=4 << 30)
    yield c
    c.close()


def _same(r, ref, tcount=True):
    assert r.hist.tolist() == ref.hist.tolist()
    assert r.hash == ref.hash
    if tcount:
        assert r.tcount.tolist() == ref.tcount.tolist()


def _small_graphs(count, seed0):
    out = []
    for s in range(count):
        n = 3 + s % 20
        p = [0.1, 0.2, 0.35, 0.5, 0.8][s % 5]
        out.append(I.gnp(n, p, seed0 + s))
    return out


def test_small_random_graphs(ctx):
    for g in _small_graphs(200, 4242):
        _same(ctx.enumerate(g), oracle.enumerate_cycles(g))


@pytest.mark.parametrize("g", [I.gnp(65, 2.6 / 65, 65), I.gnp(100, 2.4 / 100, 100), I.gnp(128, 2.4 / 128, 128),
                               I.gnp(129, 2.6 / 129, 129), I.gnp(200, 1.9 / 200, 200), I.gnp(256, 1.8 / 256, 256),
                               I.complete_bipartite(40, 40), I.wheel(200), I.cycle(250)], ids=lambda g: g.name)
def test_bitset_widths(ctx, g):
    # two- and four-word bitset rows, and the boundaries between the widths (sparse random
    # graphs much denser than these have far too many chordless paths to enumerate)
    _same(ctx.enumerate(g), oracle.enumerate_cycles(g))


@pytest.mark.parametrize("g", [I.grid(6, 6), I.grid(4, 10), I.grid(5, 6), I.grid(5, 10), I.complete_bipartite(8, 8),
                               I.cycle(100), I.wheel(100), I.complete_bipartite(50, 50), I.complete(20)],
                         ids=lambda g: g.name)
def test_table1_graphs(ctx, g):
    _same(ctx.enumerate(g), oracle.enumerate_cycles(g))


def _table1_grids():
    # k l total hash hist[4..]: totals from Table 1, histogram and hash from the oracle
    # (tests/golden/make_table1_hashes.py)
    import os
    out = {}
    for line in open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_grids.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out[(int(f[0]), int(f[1]))] = (int(f[2]), int(f[3], 16), [0, 0, 0, 0] + [int(x) for x in f[4:]])
    return out


def _same_as_table1(r, k, l):
    total, hsh, hist = _table1_grids()[(k, l)]
    got = [int(x) for x in r.hist]
    while got and got[-1] == 0:
        got.pop()
    assert r.total == total and got == hist and r.hash == hsh


def test_grid6x10_table1(ctx):
    _same_as_table1(ctx.enumerate(I.grid(6, 10)), 6, 10)


def test_wheel_with_hub_closed_form(ctx):
    # W_k: k triangles and the rim; n = 1501 with a hub of degree 1500, CSR path with
    # paths of up to 1500 vertices
    k = 1500
    r = ctx.enumerate(I.wheel(k))
    assert r.total == k + 1 and int(r.hist[3]) == k and int(r.hist[k]) == 1


@pytest.mark.parametrize("k,l,total", [(7, 10, 8136453), (8, 10, 71535910)])
def test_large_grids_table1(ctx, k, l, total):
    # the two largest synthetic rows of Table 1 (no triangles in a grid, so the total is
    # the printed #clc); the 8x10 row is the paper's count-only run
    r = ctx.enumerate(I.grid(k, l))
    assert r.total == total
    assert int(r.hist[3]) == 0 and int(r.hist[4]) == (k - 1) * (l - 1)
    _same_as_table1(r, k, l)


@pytest.mark.parametrize("max_len", [1, 2, 3, 4, 5, 8, 13])
def test_length_bound(ctx, max_len):
    for g in [I.grid(5, 5), I.gnp(40, 0.12, 3), I.wheel(12), I.gnp(150, 0.022, 9)]:
        _same(ctx.enumerate(g, max_len=max_len), oracle.enumerate_cycles(g, max_len=max_len))


def test_edge_cases(ctx):
    for g in [I.empty(0), I.empty(1), I.empty(2), I.empty(10), I.path(2), I.path(30), I.complete(3),
              I.cycle(3), I.cycle(4), I.random_tree(40, 1), I.random_unicyclic(50, 2),
              I.from_edges(9, [(0, 1), (1, 2), (2, 0), (4, 5), (5, 6), (6, 7), (7, 4)])]:
        r = ctx.enumerate(g)
        ref = oracle.enumerate_cycles(g)
        _same(r, ref)


def test_largest_n(cc, ctx):
    # n at the CSR limit (32768): the labelling's longest sequential loop, and a graph too
    # large for the shared-memory staging (rows, ids and signatures are read from global
    # memory); against the oracle with a length bound
    lim = cc.cc_get_limits()
    g = I.gnm(lim.max_n_csr, 40000, 1)
    _same(ctx.enumerate(g, max_len=8), oracle.enumerate_cycles(g, max_len=8))
    # one more vertex is refused on the host
    big = I.gnm(lim.max_n_csr + 1, 10, 1)
    s, _ = cc.cc_graph_load(ctx.handle, big.n, big.row_ptr, big.col)
    assert s == cc.CC_ERR_UNSUPPORTED
    # a long cycle: one chordless cycle of 4096 vertices, paths of up to 4095 vertices
    r = ctx.enumerate(I.cycle(4096))
    assert r.total == 1 and int(r.hist[4096]) == 1


def test_invalid_graphs(cc, ctx):
    bad = [
        (3, [0, 1, 1, 1], [1]),               # 0 -> 1 without 1 -> 0
        (2, [0, 1, 2], [0, 1]),               # self-loops
        (3, [0, 2, 3, 4], [1, 1, 0, 0]),      # duplicate neighbour
        (2, [0, 1, 2], [5, 0]),               # id out of range
        (2, [0, 2, 1], [1, 0]),               # decreasing row_ptr
    ]
    for n, rp, cl in bad:
        s, h = cc.cc_graph_load(ctx.handle, n, np.array(rp, np.uint32), np.array(cl, np.uint32))
        assert s == cc.CC_ERR_INVALID_GRAPH, (n, rp, cl, s)


def test_unsorted_rows_accepted(ctx):
    g = I.grid(4, 4)
    rp, cl = g.row_ptr.copy(), g.col.copy()
    for v in range(g.n):
        cl[rp[v]:rp[v + 1]] = cl[rp[v]:rp[v + 1]][::-1]
    g2 = I.Graph(g.n, rp, cl)
    _same(ctx.enumerate(g2), oracle.enumerate_cycles(g))


def test_csr_mode_equals_bitset_mode(cc):
    with cc.Context(frontier_bytes=1 << 30, mode=cc.CC_MODE_CSR) as c:
        for g in _small_graphs(60, 99) + [I.grid(6, 6), I.wheel(30), I.complete_bipartite(6, 7)]:
            r = c.enumerate(g)
            assert r.info.mode == cc.CC_MODE_CSR
            _same(r, oracle.enumerate_cycles(g))


def test_csr_long_paths(cc):
    # paths of more than 32 vertices take the warp-per-path CSR form: forced CSR mode on
    # graphs with long chordless cycles, cycle lists included
    with cc.Context(frontier_bytes=1 << 30, mode=cc.CC_MODE_CSR) as c:
        for g in [I.cycle(100), I.wheel(80), I.gnm(120, 135, 3)]:
            r = c.enumerate(g, cycles=True)
            ref = oracle.enumerate_cycles(g, cycles=True)
            assert r.info.mode == cc.CC_MODE_CSR and max(len(x) for x in ref.cycles) > 33
            assert sorted(r.cycles) == sorted(ref.cycles)
            _same(r, ref)
        # 58547 of the 86350 chordless cycles of the 4 x 16 grid have more than 33 vertices
        g = I.grid(4, 16)
        _same(c.enumerate(g), oracle.enumerate_cycles(g))
        # length bounds inside the long form: closings up to L', no path stored at L'
        for L in (34, 40):
            _same(c.enumerate(g, max_len=L), oracle.enumerate_cycles(g, max_len=L))


def test_cycle_lists(ctx):
    for g in _small_graphs(40, 7) + [I.grid(4, 5), I.wheel(9), I.complete(6), I.cycle(40)]:
        r = ctx.enumerate(g, cycles=True)
        ref = oracle.enumerate_cycles(g, cycles=True)
        assert sorted(r.cycles) == sorted(ref.cycles)
        _same(r, ref)


def test_cycle_list_truncation(cc, ctx):
    g = I.grid(4, 4)
    with ctx.load(g) as lg:
        s, hist, h, tc, cyc, info = cc.cc_enumerate(lg.handle, g.n, 0, True, (3, 10))
        assert s == cc.CC_ERR_TRUNCATED
        ref = oracle.enumerate_cycles(g)
        assert cyc == (ref.total, int(sum(k * int(c) for k, c in enumerate(ref.hist))))
        assert hist.tolist() == ref.hist.tolist() and h == ref.hash


@pytest.mark.parametrize("budget", [256 << 10, 1 << 20, 64 << 20])
def test_bounded_frontier_spill(cc, budget):
    # grid 7x7 peaks at 80,935 stored paths (20 bytes each, two levels live at once);
    # budgets far below that force depth-first chunks, 64 MiB does not
    g = I.grid(7, 7)
    ref = oracle.enumerate_cycles(g)
    with cc.Context(frontier_bytes=budget) as c:
        r = c.enumerate(g)
    _same(r, ref)
    assert r.info.spilled == (1 if budget <= 1 << 20 else 0)
    assert r.info.peak_bytes <= budget


def test_spill_csr(cc):
    g = I.gnm(400, 800, 5)
    ref = oracle.enumerate_cycles(g, max_len=10)
    with cc.Context(frontier_bytes=2 << 20) as c:
        r = c.enumerate(g, max_len=10)
    _same(r, ref)
    assert r.info.spilled == 1


def test_capacity_error(cc):
    # the initial triplets of K_{50,50} (up to (Delta-1)m/2 = 61250 paths) cannot fit 64 KiB
    with cc.Context(frontier_bytes=1 << 16) as c:
        with pytest.raises(cc.CCError) as e:
            c.enumerate(I.complete_bipartite(50, 50))
        assert e.value.status == cc.CC_ERR_CAPACITY
        # the context stays usable
        _same(c.enumerate(I.grid(3, 3)), oracle.enumerate_cycles(I.grid(3, 3)))


def test_barrier_timeout_reports_status(cc):
    # a poll limit of one makes the grid barrier give up at once: the call must return
    # CC_ERR_TIMEOUT (no fault, no hang) and a later call on a fresh context must work
    # (the cluster phase, which has no polled wait, is switched off so the grid runs)
    with cc.Context(spin_limit=1, flags=cc.CC_FLAG_NO_CLUSTER_PHASE) as c:
        with pytest.raises(cc.CCError) as e:
            c.enumerate(I.grid(6, 6))
        assert e.value.status == cc.CC_ERR_TIMEOUT
    with cc.Context() as c:
        _same(c.enumerate(I.grid(6, 6)), oracle.enumerate_cycles(I.grid(6, 6)))


def test_torch_workspace_and_stream(cc):
    import torch
    with cc.Context(frontier_bytes=256 << 20, use_torch=True) as c:
        g = I.gnp(50, 0.12, 1)
        _same(c.enumerate(g), oracle.enumerate_cycles(g))
    torch.cuda.synchronize()


def test_relabelling_invariance(ctx):
    g = I.gnp(45, 0.15, 17)
    perm = I.random_permutation(g.n, 5)
    a = ctx.enumerate(g, cycles=True)
    b = ctx.enumerate(I.permute(g, perm), cycles=True)
    assert a.hist.tolist() == b.hist.tolist()
    assert sorted(tuple(sorted(int(perm[v]) for v in c)) for c in a.cycles) == \
        sorted(tuple(sorted(c)) for c in b.cycles)


# ------------------------------------------------------------------ full-size workloads

def test_grid8x8_full(ctx):
    g = I.grid(8, 8)
    _same(ctx.enumerate(g), oracle.enumerate_parallel(g))


def test_gnp60_full(ctx):
    g = I.gnp(60, 0.15, 7)
    _same(ctx.enumerate(g), oracle.enumerate_parallel(g))


def test_gnm2000_len12_full(ctx):
    g = I.gnm(2000, 4000, 11)
    r = ctx.enumerate(g, max_len=12)
    assert r.info.mode == 2  # CSR path: n = 2000 does not fit the bitset rows
    _same(r, oracle.enumerate_parallel(g, max_len=12))


# ------------------------------------------------------------------ batches

def _oracle_many(graphs, max_len=0):
    import concurrent.futures as cf
    import os
    with cf.ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        return list(ex.map(lambda g: oracle.enumerate_cycles(g, max_len=max_len), graphs))


def _check_batch(graphs, refs, hist, hsh, paths):
    for i, (g, ref) in enumerate(zip(graphs, refs)):
        L = len(ref.hist) - 1
        assert hist[i, :L + 1].tolist() == ref.hist.tolist(), (i, g.name)
        assert int(hist[i, L + 1:].sum()) == 0
        assert int(hsh[i]) == ref.hash, (i, g.name)
        assert int(paths[i]) == int(ref.tcount.sum()), (i, g.name)


def test_batch_mixture(ctx):
    graphs = I.mixture(400, 31)
    hist, hsh, paths, done, info = ctx.batch(graphs, max_len=7)
    _check_batch(graphs, _oracle_many(graphs, 7), hist, hsh, paths)


def test_batch_mixture_unbounded_small(ctx):
    graphs = [g for g in I.mixture(300, 8) if g.n <= 30]
    hist, hsh, paths, done, info = ctx.batch(graphs)
    _check_batch(graphs, _oracle_many(graphs), hist, hsh, paths)


def test_batch_full_mixture_sampled(ctx):
    # the full 4096-graph mixture in one launch; every K_{a,b} against its closed form,
    # every grid and a seeded sample of the random graphs against the oracle
    graphs = I.mixture(4096, 0)
    hist, hsh, paths, done, info = ctx.batch(graphs)
    for i, g in enumerate(graphs):
        if g.meta["family"] == "kab":
            a, b = g.meta["a"], g.meta["b"]
            assert int(hist[i, 4]) == int(hist[i].sum()) == (a * (a - 1) // 2) * (b * (b - 1) // 2)
    pick = [i for i, g in enumerate(graphs) if g.meta["family"] == "grid"]
    rng = np.random.default_rng(2024)
    gnp_idx = [i for i, g in enumerate(graphs) if g.meta["family"] == "gnp"]
    pick += sorted(rng.choice(gnp_idx, 256, replace=False).tolist())
    sub = [graphs[i] for i in pick]
    _check_batch(sub, _oracle_many(sub), hist[pick], hsh[pick], paths[pick])
    # per-graph completion: inside the batch's device time; 0 for graphs without initial
    # triplets (finished by seeding), positive for graphs with a cycle of 5 or more vertices
    # (one of their triplets had children, so it was stored and expanded)
    no_paths = np.array([int(paths[i]) == 0 for i in range(len(graphs))])
    long_cycle = np.array([int(hist[i, 5:].sum()) > 0 for i in range(len(graphs))])
    assert (done[no_paths] == 0).all()
    assert (done[long_cycle] > 0).all()
    assert (done >= 0).all() and done.max() <= info.ms_proc * 1000.0 + 1.0


def test_batch_resident_set_runs(cc, ctx):
    # cc_batch_load once, cc_batch_run twice with different length bounds: each run equals
    # cc_batch_submit of the same graphs and the oracle
    graphs = I.mixture(300, 41)
    with ctx.load_batch(graphs) as bs:
        for L in (8, 6, 8):
            hist, hsh, paths, done, info = bs.run(max_len=L)
            h2, s2, p2, _, _ = ctx.batch(graphs, max_len=L)
            assert (hist == h2).all() and (hsh == s2).all() and (paths == p2).all()
            _check_batch(graphs, _oracle_many(graphs, L), hist, hsh, paths)
            assert info.ms_total >= info.ms_proc >= info.ms_engine > 0


def test_batch_set_errors(cc, ctx):
    graphs = I.mixture(8, 3)
    bad = list(graphs)
    bad[5] = I.grid(9, 9)  # 81 vertices: beyond the batch limit
    s, h, idx = cc.cc_batch_load(ctx.handle, I.pack(bad))
    assert s == cc.CC_ERR_UNSUPPORTED and idx == 5 and not h
    with ctx.load_batch(graphs) as bs:
        s, bid = cc.cc_batch_run(bs.handle, 0)
        assert s == cc.CC_OK
        s2, _ = cc.cc_batch_run(bs.handle, 0)  # one batch in flight per context
        assert s2 == cc.CC_ERR_ARG
    # freeing the set waited for its batch; the context is usable again
    hist, hsh, paths, done, info = ctx.batch(graphs)
    _check_batch(graphs, _oracle_many(graphs), hist, hsh, paths)


def test_batch_alone_equals_mixed(ctx):
    graphs = I.mixture(64, 77)
    hist, hsh, paths, done, info = ctx.batch(graphs, max_len=9)
    for i in range(0, 64, 7):
        h1, s1, p1, _, _ = ctx.batch([graphs[i]], max_len=9)
        assert h1[0].tolist() == hist[i].tolist() and s1[0] == hsh[i] and p1[0] == paths[i]
        r = ctx.enumerate(graphs[i], max_len=9)
        assert r.hist.tolist() == hist[i, :len(r.hist)].tolist() and r.hash == int(hsh[i])


def test_batch_spill(cc):
    graphs = I.mixture(48, 5)
    with cc.Context(frontier_bytes=3 << 20) as c:
        hist, hsh, paths, done, info = c.batch(graphs, max_len=8)
    assert info.spilled == 1
    _check_batch(graphs, _oracle_many(graphs, 8), hist, hsh, paths)


def test_cluster_phase_equals_grid_only(cc):
    # small levels run on one thread-block cluster before the persistent grid takes over;
    # switching that phase off must not change any result
    graphs = [I.grid(6, 6), I.grid(8, 8), I.gnp(60, 0.15, 7), I.wheel(100), I.gnp(100, 2.4 / 100, 100),
              I.complete_bipartite(8, 8)] + _small_graphs(40, 606)
    # (one level per step on both sides, so the step counts compare; a nonzero phase size
    # runs the phase for dense graphs too)
    with cc.Context(frontier_bytes=2 << 30, flags=cc.CC_FLAG_NO_FUSE, small_phase_paths=32768) as a, \
            cc.Context(frontier_bytes=2 << 30, flags=cc.CC_FLAG_NO_CLUSTER_PHASE | cc.CC_FLAG_NO_FUSE) as b:
        for g in graphs:
            ra, rb = a.enumerate(g), b.enumerate(g)
            assert ra.hist.tolist() == rb.hist.tolist() and ra.hash == rb.hash
            assert ra.tcount.tolist() == rb.tcount.tolist()
            assert ra.info.steps == rb.info.steps
            assert ra.info.launches == rb.info.launches + 1  # the cluster launch
        for g in graphs[6:]:
            _same(a.enumerate(g), oracle.enumerate_cycles(g))


def test_cluster_phase_two_level_steps(cc):
    # the cluster phase's per-lane two-level form (sparse graphs): same results as the grid
    # alone, in fewer steps; dense graphs skip the phase unless its size is given
    sparse = [I.grid(5, 5), I.grid(6, 6), I.grid(6, 7), I.grid(4, 12), I.cycle(40), I.wheel(5)]
    with cc.Context(frontier_bytes=2 << 30) as a, \
            cc.Context(frontier_bytes=2 << 30, flags=cc.CC_FLAG_NO_CLUSTER_PHASE) as b, \
            cc.Context(frontier_bytes=2 << 30, flags=cc.CC_FLAG_NO_FUSE) as u:
        for g in sparse:
            ra, rb, ru = a.enumerate(g), b.enumerate(g), u.enumerate(g)
            ref = oracle.enumerate_cycles(g)
            _same(ra, ref)
            _same(rb, ref)
            assert ra.info.launches == rb.info.launches + 1
            assert ra.info.steps <= ru.info.steps
        ra = a.enumerate(I.grid(6, 6))
        assert ra.info.steps < u.enumerate(I.grid(6, 6)).info.steps
        g = I.gnp(60, 0.15, 7)
        assert a.enumerate(g).info.launches == b.enumerate(g).info.launches


def test_trace_matches_level_counts(cc, ctx):
    g = I.grid(7, 7)
    with cc.Context(frontier_bytes=4 << 30, flags=cc.CC_FLAG_NO_FUSE) as c1:
        r = c1.enumerate(g)
        t_ns, expanded = cc.cc_get_trace(c1.handle)
    assert len(expanded) == r.info.steps
    # without spilling or two-level steps every step expands one whole level: the trace
    # lists |T_3|..|T_{L'-1}|
    nz = [int(x) for x in r.tcount if x]
    assert [int(x) for x in expanded] == nz
    assert (np.diff(t_ns.astype(np.int64)) >= 0).all()
    # with two-level steps a step expands one level or two consecutive ones
    r2 = ctx.enumerate(g)
    _, expanded2 = cc.cc_get_trace(ctx.handle)
    assert r2.tcount.tolist() == r.tcount.tolist() and r2.info.steps < r.info.steps
    i = 0
    for e in (int(x) for x in expanded2):
        if e == nz[i]:
            i += 1
        else:
            assert e == nz[i] + nz[i + 1]
            i += 2
    assert i == len(nz)


def test_two_level_steps_equal_single_levels(cc):
    # expanding a level together with its children (storing only the grandchildren) must
    # not change any result, for every bitset width and with length bounds that end a
    # two-level step on the last level
    graphs = [I.grid(6, 6), I.grid(8, 8), I.gnp(60, 0.15, 7), I.wheel(100), I.gnp(100, 2.4 / 100, 100),
              I.gnp(200, 1.9 / 200, 200), I.complete_bipartite(8, 8)] + _small_graphs(40, 909)
    with cc.Context(frontier_bytes=2 << 30) as a, \
            cc.Context(frontier_bytes=2 << 30, flags=cc.CC_FLAG_NO_FUSE) as b:
        for g in graphs:
            for L in (0, 5, 6, 9):
                ra, rb = a.enumerate(g, max_len=L), b.enumerate(g, max_len=L)
                assert ra.hist.tolist() == rb.hist.tolist() and ra.hash == rb.hash, (g.name, L)
                assert ra.tcount.tolist() == rb.tcount.tolist(), (g.name, L)
                assert ra.info.steps <= rb.info.steps
        for g in graphs[7:]:
            _same(a.enumerate(g), oracle.enumerate_cycles(g))
        _same(a.enumerate(graphs[4], max_len=9), oracle.enumerate_cycles(graphs[4], max_len=9))


# ------------------------------------------------------------------ triplet sharding

@pytest.mark.parametrize("g,L", [(I.grid(8, 8), 0), (I.gnp(60, 0.15, 7), 0), (I.gnp(100, 0.028, 7), 0),
                                 (I.gnp(200, 1.9 / 200, 200), 0), (I.gnm(2000, 4000, 11), 9), (I.grid(5, 6), 0)])
def test_enumerate_part_equals_oracle_part(ctx, g, L):
    # each part equals the oracle's part of the same triplet split, and the parts add up
    nparts = 3
    whole = oracle.enumerate_cycles(g, max_len=L)
    with ctx.load(g) as lg:
        hist = np.zeros_like(whole.hist)
        tc = np.zeros_like(whole.tcount)
        hsh = 0
        for part in range(nparts):
            r = lg.enumerate(L, part=part, nparts=nparts)
            ref = oracle.enumerate_cycles(g, max_len=L, part=part, nparts=nparts)
            _same(r, ref)
            hist += r.hist
            tc += r.tcount
            hsh = (hsh + r.hash) % 2 ** 64
        assert hist.tolist() == whole.hist.tolist() and hsh == whole.hash and tc.tolist() == whole.tcount.tolist()


def test_enumerate_part_csr_mode_and_cycles(cc):
    g = I.gnp(40, 0.12, 9)
    with cc.Context(frontier_bytes=1 << 30, mode=cc.CC_MODE_CSR) as c, c.load(g) as lg:
        allc = []
        for part in range(2):
            r = lg.enumerate(0, cycles=True, part=part, nparts=2)
            ref = oracle.enumerate_cycles(g, cycles=True, part=part, nparts=2)
            _same(r, ref)
            assert sorted(r.cycles) == sorted(ref.cycles)
            allc += r.cycles
        assert sorted(allc) == sorted(oracle.enumerate_cycles(g, cycles=True).cycles)


def test_enumerate_part_arguments(cc, ctx):
    with ctx.load(I.grid(4, 4)) as lg:
        s, *_ = cc.cc_enumerate(lg.handle, 16, 0, True, None, 2, 2)
        assert s == cc.CC_ERR_ARG
        s, *_ = cc.cc_enumerate(lg.handle, 16, 0, True, None, 1, 0)
        assert s == cc.CC_ERR_ARG
        r = lg.enumerate(0, part=0, nparts=1)
        assert r.total == oracle.enumerate_cycles(I.grid(4, 4)).total


# ------------------------------------------------------------------ niche overlap graphs (Section 5)

@pytest.mark.parametrize("n,C,seed", [(24, 0.15, 1), (39, 0.12, 2), (69, 0.25, 3), (128, 0.2, 4), (500, 0.05, 5),
                                      (2000, 0.01, 6)])
def test_niche_overlap_equals_oracle(cc, ctx, n, C, seed):
    pp, pi = I.niche_model_web(n, C, seed)
    s, rp, col = cc.cc_niche_overlap(ctx.handle, n, pp, pi)
    assert s == cc.CC_OK
    ref_rp, ref_col = oracle.niche_overlap(n, pp, pi)
    assert rp.tolist() == ref_rp.tolist() and col.tolist() == ref_col.tolist()
    if n <= 128:
        # and its chordless cycles, as the paper enumerates them
        g = I.graph_from_csr(n, rp, col)
        _same(ctx.enumerate(g), oracle.enumerate_cycles(g))


def test_niche_overlap_truncation_and_errors(cc, ctx):
    pp, pi = I.niche_model_web(60, 0.2, 9)
    s, rp, col = cc.cc_niche_overlap(ctx.handle, 60, pp, pi, col_capacity=3)
    assert s == cc.CC_ERR_TRUNCATED and int(rp[-1]) > 3
    s, rp2, col2 = cc.cc_niche_overlap(ctx.handle, 60, pp, pi)
    assert s == cc.CC_OK and rp2.tolist() == rp.tolist()
    bad = pi.copy()
    bad[0] = 60
    s, _, _ = cc.cc_niche_overlap(ctx.handle, 60, pp, bad)
    assert s == cc.CC_ERR_INVALID_GRAPH


# ------------------------------------------------------------------ host frontier (Section 6)

@pytest.mark.parametrize("g,L,arena", [(I.grid(7, 7), 0, 256 << 10), (I.gnm(400, 800, 9), 11, 512 << 10),
                                       (I.gnp(60, 0.15, 7), 0, 1 << 20)])
def test_host_frontier_equals_oracle(cc, g, L, arena):
    # a frontier far too small for the graph: frames move to pinned host memory and back,
    # and the result is still the oracle's.  (How often frames move depends on the order in
    # which a level's records were written, which the slot atomics leave free, so the test
    # takes arenas small enough that some move in every run.)
    ref = oracle.enumerate_cycles(g, max_len=L)
    with cc.Context(frontier_bytes=arena, host_frontier_bytes=2 << 30) as c, c.load(g) as lg:
        r = lg.enumerate(L)
        _same(r, ref)
        assert r.info.host_offloads > 0 and r.info.spilled == 1
        assert r.info.peak_bytes <= arena
        r2 = lg.enumerate(L)  # a second call (no CUDA graph with a host frontier)
        _same(r2, ref)
        assert r2.info.replayed == 0


def test_host_frontier_too_small_reports_capacity(cc):
    # A 256 KiB arena cannot hold grid 7x7's larger levels, so the engine stops to move
    # frames to the host at least once, and that move always includes the frame being
    # expanded (it has records left).  16 bytes of host frontier hold no packed record (20
    # bytes), so the first move fails.  (With 64 KiB the outcome depended on how large the
    # waiting frames happened to be, which varies with the order of the records.)
    g = I.grid(7, 7)
    with cc.Context(frontier_bytes=256 << 10, host_frontier_bytes=16) as c, c.load(g) as lg:
        s, *_ = cc.cc_enumerate(lg.handle, g.n, 0)
        assert s == cc.CC_ERR_CAPACITY
        # the context stays usable
    with cc.Context(frontier_bytes=1 << 30) as c:
        _same(c.enumerate(g), oracle.enumerate_cycles(g))


# ------------------------------------------------------------------ edge cases of the newer entry points

def test_host_frontier_with_cycle_lists(cc):
    # the host frontier moves CSR frames (cycle lists force CSR records); the listed cycles
    # are the oracle's
    g = I.grid(7, 7)
    ref = oracle.enumerate_cycles(g, cycles=True)
    with cc.Context(frontier_bytes=128 << 10, host_frontier_bytes=1 << 30) as c, c.load(g) as lg:
        r = lg.enumerate(0, cycles=True)
        _same(r, ref)
        assert sorted(r.cycles) == sorted(ref.cycles)
        assert r.info.host_offloads > 0


@pytest.mark.parametrize("L", [3, 4, 5])
def test_enumerate_part_short_bounds_and_empty_parts(ctx, L):
    # more parts than triplets: some parts are empty; short length bounds
    g = I.wheel(5)
    nparts = 64
    whole = oracle.enumerate_cycles(g, max_len=L)
    with ctx.load(g) as lg:
        tot = np.zeros_like(whole.hist)
        hsh = 0
        empty = 0
        for part in range(nparts):
            r = lg.enumerate(L, part=part, nparts=nparts)
            _same(r, oracle.enumerate_cycles(g, max_len=L, part=part, nparts=nparts))
            tot += r.hist
            hsh = (hsh + r.hash) % 2 ** 64
            empty += r.total == 0
        assert tot.tolist() == whole.hist.tolist() and hsh == whole.hash and empty > 0


def test_batch_degenerate_graphs(cc, ctx):
    # graphs without cycles, without edges, with fewer than 3 vertices, and length bounds 3
    graphs = [I.empty(1), I.empty(2), I.path(2), I.empty(5), I.path(7), I.random_tree(20, 3), I.cycle(3),
              I.complete(4), I.grid(3, 3)]
    for L in (0, 3, 4):
        hist, hsh, paths, done, info = ctx.batch(graphs, max_len=L)
        _check_batch(graphs, _oracle_many(graphs, L), hist, hsh, paths)


def test_niche_overlap_small_webs(cc, ctx):
    for n, lists in [(1, [[0]]), (2, [[], []]), (2, [[0], [0]]), (3, [[0], [0], [0]]), (4, [[], [], [], []])]:
        ptr = np.zeros(n + 1, dtype=np.uint32)
        ptr[1:] = np.cumsum([len(x) for x in lists])
        idx = np.array([z for x in lists for z in x], dtype=np.uint32)
        s, rp, col = cc.cc_niche_overlap(ctx.handle, n, ptr, idx)
        assert s == cc.CC_OK
        ref_rp, ref_col = oracle.niche_overlap(n, ptr, idx)
        assert rp.tolist() == ref_rp.tolist() and col.tolist() == ref_col.tolist()
