"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check is chosen so that a plausible mistake in the oracle (a dropped chord test,
a wrong label comparison, an off-by-one in the length bound, a wrong hash constant)
fails at least one of them:
  * counts printed in Table 1 of the paper (tests/golden/table1_synthetic.txt);
  * closed forms: C_n, K_n, K_{a,b}, wheels, grids, trees, unicyclic graphs (Section 2);
  * the definition itself, by brute force over vertex subsets, on hundreds of seeded graphs;
  * an independent library enumerator (networkx) where it is installed;
  * the level sets T_t against their definition by brute force over vertex sequences;
  * degree labellings worked by hand (tests/golden/degree_labeling.txt);
  * the published SplitMix64 sequence behind the cycle hash (tests/golden/splitmix64.txt).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1410_4876_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ------------------------------------------------------------------ hash

def test_splitmix64_known_answer():
    lines = [l for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if l.strip() and not l.startswith("#")]
    seed = int(lines[0].split()[1])
    expect = [int(x) for x in lines[1:]]
    got, s = [], seed
    for _ in expect:
        v, s = oracle.splitmix64_next(s)
        got.append(v)
    assert got == expect


def test_vertex_hash_is_splitmix_draw():
    # r(v) is the SplitMix64 output for state (v + 1) * GAMMA, i.e. draw v of the seed-0 stream.
    s = 0
    for v in range(50):
        out, s = oracle.splitmix64_next(s)
        assert oracle.vertex_hash(v) == out


def test_cycle_hash_is_set_function():
    c = [5, 9, 2, 7]
    h = oracle.cycle_hash(c)
    for perm in itertools.permutations(c):
        assert oracle.cycle_hash(list(perm)) == h
    assert oracle.cycle_hash([5, 9, 2]) != h
    assert oracle.cycle_hash([5, 9, 2, 8]) != h


def _splitmix_draw(state: int) -> int:
    return oracle.splitmix64_next(state)[0]


GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


@pytest.mark.parametrize("cyc", [(0, 1, 2), (3, 5, 8, 9), (7, 1, 4, 0, 12), tuple(range(10, 22))])
def test_cycle_hash_from_the_published_stream(cyc):
    # h(C) = mix(sum r(v) + |C| * GAMMA) with r(v) = draw v (0-based) of the seed-0
    # SplitMix64 stream.  Both sides are built here from the generator alone (pinned by
    # the published output sequence above): r(v) by drawing v + 1 times from state 0, and
    # h(C) as the next draw from the state sum r(v) + (|C| - 1) GAMMA, since a draw first
    # adds GAMMA to the state.  A dropped, doubled or mis-scaled length term fails here.
    r = {}
    for v in cyc:
        s, out = 0, None
        for _ in range(v + 1):
            out, s = oracle.splitmix64_next(s)
        r[v] = out
    k = len(cyc)
    state = (sum(r.values()) + (k - 1) * GAMMA) & MASK
    assert oracle.cycle_hash(list(cyc)) == _splitmix_draw(state)
    # the length term is really there: the same draw without it differs
    assert oracle.cycle_hash(list(cyc)) != _splitmix_draw((sum(r.values()) - GAMMA) & MASK)


def test_graph_hash_of_single_cycles():
    # a graph that is one chordless cycle hashes to that cycle's h(C), built from the stream
    for k in (3, 4, 7):
        g = I.cycle(k)
        s, rsum = 0, 0
        for _ in range(k):
            out, s = oracle.splitmix64_next(s)
            rsum += out
        expect = _splitmix_draw((rsum + (k - 1) * GAMMA) & MASK)
        assert oracle.enumerate_cycles(g).hash == expect
        assert oracle.bruteforce(g).hash == expect


# ------------------------------------------------------------------ degree labelling

def _golden_labelings():
    out = []
    for line in open(os.path.join(GOLDEN, "degree_labeling.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        name, n, edges, labels = [x.strip() for x in line.split("|")]
        e = [tuple(int(v) for v in x.split("-")) for x in edges.split()]
        out.append((name, int(n), e, [int(x) for x in labels.split()]))
    return out


@pytest.mark.parametrize("name,n,edges,labels", _golden_labelings())
def test_degree_labeling_golden(name, n, edges, labels):
    g = I.from_edges(n, edges)
    assert oracle.degree_labeling(g).tolist() == labels


def _check_labeling_property(g, lab):
    # Section 2: l(u_i) = i where u_i has minimum degree in G_i = G - {u_1..u_{i-1}};
    # ties go to the smallest id.
    order = np.argsort(lab)
    alive = set(range(g.n))
    adj = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    for u in order.tolist():
        degs = {v: len(adj[v] & alive) for v in alive}
        dmin = min(degs.values())
        assert degs[u] == dmin
        assert u == min(v for v in alive if degs[v] == dmin)
        alive.remove(u)


@pytest.mark.parametrize("seed", range(20))
def test_degree_labeling_property(seed):
    g = I.gnp(12 + seed % 7, 0.3, seed)
    lab = oracle.degree_labeling(g)
    assert sorted(lab.tolist()) == list(range(1, g.n + 1))
    _check_labeling_property(g, lab)


# ------------------------------------------------------------------ Table 1

def _table1(speed):
    rows = []
    for line in open(os.path.join(GOLDEN, "table1_synthetic.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        fam, args, n, m, dmax, c3, clc, sp = line.split()
        if sp != speed:
            continue
        a = tuple(int(x) for x in args.split(","))
        rows.append((fam, a, int(n), int(m), int(dmax), int(c3), int(clc)))
    return rows


def _family(fam, a):
    return {"cycle": I.cycle, "wheel": I.wheel, "kab": I.complete_bipartite, "grid": I.grid}[fam](*a)


def _check_table1(fam, a, n, m, dmax, c3, clc):
    g = _family(fam, a)
    assert (g.n, g.m, g.max_degree) == (n, m, dmax)
    r = oracle.enumerate_cycles(g)
    assert int(r.hist[3]) == c3
    assert r.total - int(r.hist[3]) == clc


@pytest.mark.parametrize("fam,a,n,m,dmax,c3,clc", _table1("fast"))
def test_table1(fam, a, n, m, dmax, c3, clc):
    _check_table1(fam, a, n, m, dmax, c3, clc)


@pytest.mark.slow
@pytest.mark.parametrize("fam,a,n,m,dmax,c3,clc", _table1("slow"))
def test_table1_slow(fam, a, n, m, dmax, c3, clc):
    _check_table1(fam, a, n, m, dmax, c3, clc)


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", [3, 4, 5, 7, 16, 33, 64, 65, 130])
def test_cycle_graph(n):
    r = oracle.enumerate_cycles(I.cycle(n))
    assert r.total == 1 and int(r.hist[n]) == 1
    # one chordless path of every length 3..n-1 grows around the cycle
    assert r.tcount[3:n].tolist() == [1] * (n - 3)


@pytest.mark.parametrize("n", [3, 4, 5, 8, 12])
def test_complete_graph(n):
    r = oracle.enumerate_cycles(I.complete(n))
    assert int(r.hist[3]) == math.comb(n, 3) and r.total == math.comb(n, 3)
    assert int(r.tcount.sum()) == 0


@pytest.mark.parametrize("a,b", [(2, 2), (2, 5), (3, 3), (4, 7), (8, 8), (6, 2)])
def test_complete_bipartite(a, b):
    r = oracle.enumerate_cycles(I.complete_bipartite(a, b))
    assert int(r.hist[4]) == math.comb(a, 2) * math.comb(b, 2) == r.total


@pytest.mark.parametrize("n", [4, 5, 9, 40])
def test_wheel(n):
    r = oracle.enumerate_cycles(I.wheel(n))
    assert int(r.hist[3]) == n and int(r.hist[n]) == 1 and r.total == n + 1


@pytest.mark.parametrize("k,l", [(2, 2), (2, 7), (3, 3), (3, 5), (4, 4)])
def test_grid_squares(k, l):
    r = oracle.enumerate_cycles(I.grid(k, l))
    assert int(r.hist[4]) == (k - 1) * (l - 1)
    if (k, l) == (3, 3):
        assert r.total == 5 and int(r.hist[8]) == 1
    if k == 2:
        # a ladder: any cycle through two non-neighbouring rungs has the rungs between
        # them as chords, so the squares are the only chordless cycles
        assert r.total == l - 1


@pytest.mark.parametrize("seed", range(10))
def test_tree_has_no_triplets(seed):
    g = I.random_tree(5 + 3 * seed, seed)
    r = oracle.enumerate_cycles(g)
    assert r.total == 0 and int(r.tcount.sum()) == 0 and oracle.triplet_count(g) == 0


@pytest.mark.parametrize("seed", range(10))
def test_unicyclic_has_one_triplet(seed):
    # Section 2: a graph with a unique cycle has |T(G)| = 1 (or the cycle is a triangle)
    g = I.random_unicyclic(6 + 3 * seed, seed)
    r = oracle.enumerate_cycles(g)
    assert r.total == 1
    assert oracle.triplet_count(g) == (0 if int(r.hist[3]) == 1 else 1)


@pytest.mark.parametrize("seed", range(10))
def test_triplet_bound(seed):
    # Section 2: |T(G)| <= (Delta - 1) * m / 2
    g = I.gnp(30, 0.2, seed)
    assert oracle.triplet_count(g) <= (g.max_degree - 1) * g.m / 2


# ------------------------------------------------------------------ brute force

def _small_graphs(count, seed0=0):
    out = []
    for s in range(count):
        n = 4 + s % 11
        p = [0.15, 0.3, 0.5, 0.7][s % 4]
        out.append(I.gnp(n, p, seed0 + s))
    return out


@pytest.mark.parametrize("chunk", range(6))
def test_algorithm1_equals_definition(chunk):
    for g in _small_graphs(60, 1000 * chunk):
        a = oracle.enumerate_cycles(g, cycles=True)
        b = oracle.bruteforce(g, cycles=True)
        assert a.hist.tolist() == b.hist.tolist(), g.name
        assert a.hash == b.hash, g.name
        assert sorted(a.cycles) == sorted(b.cycles), g.name
        assert len(set(a.cycles)) == len(a.cycles)  # each cycle exactly once
        assert sum(oracle.cycle_hash(c) for c in b.cycles) % 2 ** 64 == b.hash


@pytest.mark.parametrize("max_len", [1, 2, 3, 4, 5, 7])
def test_length_bound_equals_definition(max_len):
    for g in _small_graphs(40, 77):
        a = oracle.enumerate_cycles(g, max_len=max_len)
        b = oracle.bruteforce(g, max_len=max_len)
        assert a.hist.tolist() == b.hist.tolist() and a.hash == b.hash


def test_named_small_graphs_equal_definition():
    for g in [I.grid(3, 4), I.grid(4, 4), I.complete_bipartite(3, 4), I.wheel(7), I.complete(6),
              I.cycle(9), I.path(6), I.empty(5), I.grid(2, 9), I.complete_bipartite(2, 8)]:
        a = oracle.enumerate_cycles(g, cycles=True)
        b = oracle.bruteforce(g, cycles=True)
        assert sorted(a.cycles) == sorted(b.cycles) and a.hash == b.hash


def _check_canonical_order(g, cycles):
    """Canonical ordered form (cycle lists): the smallest id first, then towards the
    smaller of its two cycle neighbours; consecutive entries (and last-first) are edges."""
    edges = {(int(a), int(b)) for a, b in g.edges().tolist()}
    edges |= {(b, a) for a, b in edges}
    for c in cycles:
        k = len(c)
        assert k >= 3
        assert c[0] == min(c), c
        assert c[1] < c[-1], c
        assert len(set(c)) == k, c
        for i in range(k):
            assert (c[i], c[(i + 1) % k]) in edges, c


@pytest.mark.parametrize("chunk", range(3))
def test_cycle_lists_in_canonical_order(chunk):
    graphs = _small_graphs(40, 3000 + 100 * chunk)
    if chunk == 0:
        graphs += [I.grid(3, 4), I.grid(4, 4), I.complete_bipartite(3, 4), I.wheel(7), I.complete(6),
                   I.cycle(9), I.grid(2, 9), I.complete_bipartite(2, 8)]
    for g in graphs:
        _check_canonical_order(g, oracle.enumerate_cycles(g, cycles=True).cycles)
        _check_canonical_order(g, oracle.bruteforce(g, cycles=True).cycles)


def test_canonical_order_worked_examples():
    # worked by hand: the 6-cycle 0-1-2-3-4-5 renamed so that the smallest id (1) sits
    # in the middle of the input order and its smaller neighbour lies "backwards"
    g = I.from_edges(8, [(7, 4), (4, 1), (1, 6), (6, 2), (2, 5), (5, 7)])
    assert oracle.enumerate_cycles(g, cycles=True).cycles == [(1, 4, 7, 5, 2, 6)]
    assert oracle.bruteforce(g, cycles=True).cycles == [(1, 4, 7, 5, 2, 6)]
    # the 4-cycle 3-0-2-1: 0's neighbours are 3 and 2, so 0, 2, 1, 3
    g = I.from_edges(4, [(3, 0), (0, 2), (2, 1), (1, 3)])
    assert oracle.enumerate_cycles(g, cycles=True).cycles == [(0, 2, 1, 3)]
    assert oracle.bruteforce(g, cycles=True).cycles == [(0, 2, 1, 3)]


def test_networkx_enumerator():
    nx = pytest.importorskip("networkx")
    if not hasattr(nx, "chordless_cycles"):
        pytest.skip("networkx without chordless_cycles")
    for g in _small_graphs(40, 555) + [I.grid(4, 4), I.wheel(6), I.complete_bipartite(3, 3)]:
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        G.add_edges_from(g.edges().tolist())
        ref = sorted(tuple(sorted(c)) for c in nx.chordless_cycles(G))
        a = oracle.enumerate_cycles(g, cycles=True)
        assert sorted(tuple(sorted(c)) for c in a.cycles) == ref


def _level_sets_by_definition(g, lab, L):
    """T_t by its definition: induced paths <v_1..v_t> (no edge between non-consecutive
    vertices) with l(v_2) minimal and l(v_1) < l(v_3), for 3 <= t < L."""
    adj = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    counts = [0] * (L + 1)
    for t in range(3, L):
        for seq in itertools.permutations(range(g.n), t):
            if any(seq[i + 1] not in adj[seq[i]] for i in range(t - 1)):
                continue
            if any(seq[j] in adj[seq[i]] for i in range(t) for j in range(i + 2, t)):
                continue
            if min(lab[v] for v in seq) != lab[seq[1]] or not lab[seq[0]] < lab[seq[2]]:
                continue
            counts[t] += 1
    return counts


@pytest.mark.parametrize("seed", range(8))
def test_level_counts_equal_definition(seed):
    g = [I.gnp(7, 0.45, seed), I.grid(2, 4), I.wheel(5), I.complete_bipartite(3, 3),
         I.gnp(8, 0.35, 100 + seed), I.cycle(7), I.grid(3, 3), I.gnp(8, 0.25, 200 + seed)][seed]
    lab = oracle.degree_labeling(g)
    r = oracle.enumerate_cycles(g)
    assert r.tcount.tolist() == _level_sets_by_definition(g, lab, g.n)


@pytest.mark.parametrize("seed", range(12))
def test_relabelling_invariance(seed):
    # Section 2: the labelling fixes each cycle's orientation uniquely for ANY bijection,
    # so renaming vertices (which changes the tie-breaks of the degree labelling) maps the
    # cycle set onto itself.
    g = I.gnp(18, 0.25, seed)
    perm = I.random_permutation(g.n, seed + 1000)
    gp = I.permute(g, perm)
    a = oracle.enumerate_cycles(g, cycles=True)
    b = oracle.enumerate_cycles(gp, cycles=True)
    assert a.hist.tolist() == b.hist.tolist()
    mapped = sorted(tuple(sorted(int(perm[v]) for v in c)) for c in a.cycles)
    assert mapped == sorted(tuple(sorted(c)) for c in b.cycles)


@pytest.mark.parametrize("nparts", [2, 3, 7])
def test_parts_add_up(nparts):
    for g, L in [(I.gnp(30, 0.2, 5), 0), (I.gnp(24, 0.35, 6), 0), (I.grid(4, 5), 0), (I.gnp(40, 0.15, 8), 9)]:
        whole = oracle.enumerate_cycles(g, max_len=L)
        parts = [oracle.enumerate_cycles(g, max_len=L, part=p, nparts=nparts) for p in range(nparts)]
        assert sum(p.hist for p in parts).tolist() == whole.hist.tolist()
        assert sum(p.tcount for p in parts).tolist() == whole.tcount.tolist()
        assert sum(p.hash for p in parts) % 2 ** 64 == whole.hash
        # a real split: no part holds everything (these graphs have many triplets)
        assert all(p.total < whole.total for p in parts)


@pytest.mark.parametrize("chunk", range(2))
def test_parts_partition_the_definition(chunk):
    # the parts' cycle lists are disjoint and together equal the brute-force cycle set
    for g in _small_graphs(30, 7000 + 100 * chunk):
        ref = sorted(oracle.bruteforce(g, cycles=True).cycles)
        got = []
        for p in range(3):
            got += oracle.enumerate_cycles(g, cycles=True, part=p, nparts=3).cycles
        assert sorted(got) == ref


# ------------------------------------------------------------------ niche overlap graph (Section 5)

def _web(n, prey_lists):
    ptr = np.zeros(n + 1, dtype=np.uint32)
    ptr[1:] = np.cumsum([len(p) for p in prey_lists])
    idx = np.array([z for p in prey_lists for z in p], dtype=np.uint32)
    return ptr, idx


def _edges(rp, col):
    return {(x, int(y)) for x in range(len(rp) - 1) for y in col[rp[x]:rp[x + 1]]}


def test_niche_overlap_shared_prey_gives_a_clique():
    # one prey (0) eaten by species 1..k: the k predators overlap pairwise (K_k); the prey
    # itself overlaps with nobody
    k = 6
    rp, col = oracle.niche_overlap(k + 1, *_web(k + 1, [[]] + [[0]] * k))
    assert _edges(rp, col) == {(x, y) for x in range(1, k + 1) for y in range(1, k + 1) if x != y}


def test_niche_overlap_food_chain_is_empty():
    # a food chain (species i eats i + 1): every prey has a single predator
    n = 9
    rp, col = oracle.niche_overlap(n, *_web(n, [[i + 1] for i in range(n - 1)] + [[]]))
    assert rp.tolist() == [0] * (n + 1) and col.size == 0


def test_niche_overlap_worked_example():
    # worked by hand: 0 eats 3, 4; 1 eats 4; 2 eats 5; 3 eats itself and 5; 4, 5 basal;
    # 6 eats 3.  Prey 3 has predators 0, 3, 6 (overlaps 0-3, 0-6, 3-6), prey 4 has 0, 1
    # (0-1), prey 5 has 2, 3 (2-3)
    rp, col = oracle.niche_overlap(7, *_web(7, [[3, 4], [4], [5], [3, 5], [], [], [3]]))
    und = {(0, 1), (0, 3), (0, 6), (3, 6), (2, 3)}
    assert _edges(rp, col) == und | {(b, a) for a, b in und}
    assert all((np.diff(col[rp[x]:rp[x + 1]].astype(np.int64)) > 0).all() for x in range(7))


def test_niche_model_overlap_graphs_are_simple_and_symmetric():
    for n, C, seed in [(24, 0.15, 1), (69, 0.25, 2), (128, 0.2, 3)]:
        rp, col = oracle.niche_overlap(n, *I.niche_model_web(n, C, seed))
        e = _edges(rp, col)
        assert all((y, x) in e and x != y for x, y in e)
        g = I.graph_from_csr(n, rp, col)
        assert g.m == len(e) // 2
