"""Seeded synthetic graph generators (inputs only: no enumeration arithmetic).

Every graph is returned as a CSR pair ``(row_ptr, col)`` of ``uint32`` arrays with
``row_ptr`` of length n+1, each row sorted ascending, every undirected edge stored
in both rows, no self-loops and no duplicates (a finite undirected simple graph,
Section 1 of the paper).

Random draws use SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; finaliser
constants of Vigna's public-domain ``splitmix64.c``) as a counter-based
generator: draw ``i`` (0-based) of a stream with key ``k`` is
``mix(k + (i + 1) * GAMMA)``, and a uniform double is ``(x >> 11) * 2**-53``.
The exact draw procedure of each generator is stated in its docstring so that
any other implementation can reproduce the same graph bit for bit.

The synthetic families follow the shapes of the paper's third workload group
(cycle, wheel, complete bipartite graphs and grids, Section 5 and Table 1) plus
the seeded random graphs and mixtures of the benchmark configurations.

This module is shared by the CPU oracle's tests and by the CUDA path's tests
and benchmark; it holds no part of the enumeration method.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO53 = float(2.0 ** -53)


def mix(z):
    """SplitMix64 output finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream(key: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of the SplitMix64 stream with this key."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix(np.uint64(key) + i * GAMMA)


def uniform(key: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the stream (53 high bits of each draw)."""
    return (stream(key, count, start) >> np.uint64(11)).astype(np.float64) * _TWO53


def seed_key(seed: int) -> int:
    """Stream key of an integer seed: the first SplitMix64 output for that seed."""
    return int(stream(int(seed) & 0xFFFFFFFFFFFFFFFF, 1)[0])


def sub_key(key: int, index: int) -> int:
    """Key of the ``index``-th child stream of ``key`` (draw ``index`` of key's stream
    passed once more through the finaliser)."""
    return int(mix(stream(key, 1, index))[0])


@dataclass
class Graph:
    """A simple undirected graph in CSR form (uint32 row offsets and neighbours)."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1]) // 2

    @property
    def max_degree(self) -> int:
        if self.n == 0:
            return 0
        return int(np.max(np.diff(self.row_ptr.astype(np.int64))))

    def edges(self) -> np.ndarray:
        """Edges (u, v) with u < v, as an (m, 2) int64 array."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr.astype(np.int64)))
        cols = self.col.astype(np.int64)
        keep = rows < cols
        return np.stack([rows[keep], cols[keep]], axis=1)


def from_edges(n: int, edges, name: str = "", meta: dict | None = None) -> Graph:
    """CSR of an undirected simple graph from (u, v) pairs (either orientation).

    Raises ValueError on a self-loop, a duplicate edge or an id outside [0, n)."""
    e = np.asarray(list(edges) if not isinstance(edges, np.ndarray) else edges, dtype=np.int64)
    e = e.reshape(-1, 2)
    if e.size and (e.min() < 0 or e.max() >= n):
        raise ValueError("vertex id out of range")
    if np.any(e[:, 0] == e[:, 1]):
        raise ValueError("self-loop")
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    keys = lo * max(n, 1) + hi
    if np.unique(keys).size != keys.size:
        raise ValueError("duplicate edge")
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return Graph(n, row_ptr.astype(np.uint32), dst.astype(np.uint32), name, meta or {})


# ---------------------------------------------------------------- named families

def grid(k: int, l: int) -> Graph:
    """k x l grid graph, vertex id = r * l + c (row-major), edges to the right and below."""
    e = []
    for r in range(k):
        for c in range(l):
            v = r * l + c
            if c + 1 < l:
                e.append((v, v + 1))
            if r + 1 < k:
                e.append((v, v + l))
    return from_edges(k * l, e, f"grid{k}x{l}", {"family": "grid", "k": k, "l": l})


def complete_bipartite(a: int, b: int) -> Graph:
    """K_{a,b}: parts [0, a) and [a, a + b)."""
    e = [(i, a + j) for i in range(a) for j in range(b)]
    return from_edges(a + b, e, f"K{a},{b}", {"family": "kab", "a": a, "b": b})


def complete(n: int) -> Graph:
    e = [(i, j) for i in range(n) for j in range(i + 1, n)]
    return from_edges(n, e, f"K{n}", {"family": "complete", "n": n})


def cycle(n: int) -> Graph:
    """C_n on vertices 0..n-1 (n >= 3)."""
    e = [(i, (i + 1) % n) for i in range(n)]
    return from_edges(n, e, f"C{n}", {"family": "cycle", "n": n})


def path(n: int) -> Graph:
    e = [(i, i + 1) for i in range(n - 1)]
    return from_edges(n, e, f"P{n}", {"family": "path", "n": n})


def wheel(n: int) -> Graph:
    """Wheel with n rim vertices 0..n-1 (a cycle) and hub n joined to all of them."""
    e = [(i, (i + 1) % n) for i in range(n)] + [(i, n) for i in range(n)]
    return from_edges(n + 1, e, f"Wheel{n}", {"family": "wheel", "n": n})


def empty(n: int) -> Graph:
    return from_edges(n, np.zeros((0, 2), dtype=np.int64), f"E{n}", {"family": "empty"})


# ---------------------------------------------------------------- seeded random graphs

def gnp(n: int, p: float, seed: int) -> Graph:
    """Erdos-Renyi G(n, p).

    Pairs (i, j), i < j, are taken in lexicographic order; pair number e (0-based)
    is an edge iff uniform draw e of the stream ``seed_key(seed)`` is < p."""
    iu, ju = np.triu_indices(n, k=1)
    u = uniform(seed_key(seed), iu.size)
    keep = u < p
    return from_edges(n, np.stack([iu[keep], ju[keep]], axis=1), f"gnp{n}_{p}_{seed}",
                      {"family": "gnp", "n": n, "p": p, "seed": seed})


def gnm(n: int, m: int, seed: int) -> Graph:
    """Uniform G(n, m) by rejection.

    Draws come in pairs from the stream ``seed_key(seed)``: pair q gives
    i = floor(u_{2q} * n), j = floor(u_{2q+1} * n); the pair is skipped if i == j or
    the edge {i, j} was already taken; draws continue until m edges are taken."""
    if m > n * (n - 1) // 2:
        raise ValueError("m too large")
    key = seed_key(seed)
    taken = set()
    edges = []
    start = 0
    while len(edges) < m:
        batch = max(2 * (m - len(edges)) * 2, 64)
        u = uniform(key, batch, start)
        start += batch
        ij = np.floor(u * n).astype(np.int64).reshape(-1, 2)
        for i, j in ij:
            if i == j:
                continue
            a, b = (i, j) if i < j else (j, i)
            if (a, b) in taken:
                continue
            taken.add((a, b))
            edges.append((a, b))
            if len(edges) == m:
                break
    return from_edges(n, edges, f"gnm{n}_{m}_{seed}", {"family": "gnm", "n": n, "m": m, "seed": seed})


def random_tree(n: int, seed: int) -> Graph:
    """Random recursive tree: vertex v >= 1 attaches to floor(u_{v-1} * v)."""
    u = uniform(seed_key(seed), max(n - 1, 0))
    e = [(v, int(np.floor(u[v - 1] * v))) for v in range(1, n)]
    return from_edges(n, e, f"tree{n}_{seed}", {"family": "tree", "n": n, "seed": seed})


def random_unicyclic(n: int, seed: int) -> Graph:
    """A random tree plus one extra edge that closes exactly one cycle (n >= 3).

    The extra edge joins the two vertices given by draws 0 and 1 of sub-stream 1,
    moved on to the next pair until the pair is a non-edge of the tree."""
    t = random_tree(n, seed)
    e = {tuple(x) for x in t.edges().tolist()}
    key = sub_key(seed_key(seed), 1)
    q = 0
    while True:
        u = uniform(key, 2, 2 * q)
        i, j = int(u[0] * n), int(u[1] * n)
        q += 1
        a, b = min(i, j), max(i, j)
        if a != b and (a, b) not in e:
            e.add((a, b))
            break
    return from_edges(n, sorted(e), f"unicyclic{n}_{seed}", {"family": "unicyclic", "n": n, "seed": seed})


def permute(g: Graph, perm: Sequence[int]) -> Graph:
    """Relabel vertex v as perm[v]."""
    perm = np.asarray(perm, dtype=np.int64)
    e = g.edges()
    return from_edges(g.n, perm[e], g.name + "_perm", dict(g.meta, permuted=True))


def random_permutation(n: int, seed: int) -> np.ndarray:
    """Permutation of 0..n-1: vertices sorted by their uniform draw (ties by id)."""
    u = uniform(seed_key(seed), n)
    return np.argsort(u, kind="stable").argsort(kind="stable")


# ---------------------------------------------------------------- mixtures

def mixture_spec(index: int, seed: int) -> Tuple[str, tuple]:
    """Member ``index`` of the batch mixture with this seed.

    Stream ``sub_key(seed_key(seed), index)`` draws u0..u3:
      u0 < 0.5  -> Erdos-Renyi G(n, p), n = 16 + floor(u1 * 49) (uniform in [16, 64]),
                   p = 0.08 + 0.22 * u2, graph seed = floor(u3 * 2**31);
      u0 < 0.8  -> grid k x l, k = 3 + floor(u1 * 4), l = 3 + floor(u2 * 4) (in [3, 6]);
      otherwise -> K_{a,b}, a = 2 + floor(u1 * 7), b = 2 + floor(u2 * 7) (in [2, 8])."""
    u = uniform(sub_key(seed_key(seed), index), 4)
    if u[0] < 0.5:
        return "gnp", (16 + int(u[1] * 49), 0.08 + 0.22 * float(u[2]), int(u[3] * 2 ** 31))
    if u[0] < 0.8:
        return "grid", (3 + int(u[1] * 4), 3 + int(u[2] * 4))
    return "kab", (2 + int(u[1] * 7), 2 + int(u[2] * 7))


def make(kind: str, args: tuple) -> Graph:
    if kind == "gnp":
        return gnp(*args)
    if kind == "grid":
        return grid(*args)
    if kind == "kab":
        return complete_bipartite(*args)
    raise ValueError(kind)


def mixture(count: int, seed: int) -> List[Graph]:
    """``count`` graphs of the batch mixture (see ``mixture_spec``)."""
    return [make(*mixture_spec(i, seed)) for i in range(count)]


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: gaps -ln(1 - u_i) / rate from
    the stream ``seed_key(seed)``, kept while the running sum is < duration."""
    key = seed_key(seed)
    out = []
    tnow, start = 0.0, 0
    while True:
        u = uniform(key, 4096, start)
        start += 4096
        gaps = -np.log1p(-u) / rate
        times = tnow + np.cumsum(gaps)
        inside = times < duration
        out.append(times[inside])
        if not inside.all():
            break
        tnow = float(times[-1])
    return np.concatenate(out)


def serving_request(index: int, seed: int) -> Tuple[str, tuple]:
    """Request ``index`` of the serving stream: with draw u0 of stream
    ``sub_key(seed_key(seed), index)``, u0 < 0.05 gives an 8 x 8 grid, otherwise
    member ``index`` of the batch mixture with the same seed."""
    u0 = float(uniform(sub_key(seed_key(seed), index), 1)[0])
    if u0 < 0.05:
        return "grid", (8, 8)
    return mixture_spec(index, seed + 1)


# ---------------------------------------------------------------- food webs

def niche_model_web(n: int, connectance: float, seed: int):
    """A seeded food web of the niche model (Williams and Martinez, Nature 2000), the
    usual synthetic stand-in for measured food webs like those of the paper's first group.
    Returns (prey_ptr, prey_idx): species x feeds on prey_idx[prey_ptr[x] .. prey_ptr[x+1])
    (ascending; cannibalism allowed).

    Stream ``seed_key(seed)`` draws 3 uniforms per species i (draws 3i, 3i+1, 3i+2): niche
    value v_i = u0; feeding range r_i = v_i * (1 - (1 - u1) ** (1 / beta)) with
    beta = 1 / (2 C) - 1 (a Beta(1, beta) draw by its inverse CDF); range centre
    c_i = r_i / 2 + u2 * (v_i - r_i / 2).  Species i eats every j with
    c_i - r_i / 2 <= v_j <= c_i + r_i / 2.  The species with the smallest niche value gets
    r = 0 (a basal species), as in the model."""
    u = uniform(seed_key(seed), 3 * n).reshape(n, 3)
    beta = 1.0 / (2.0 * connectance) - 1.0
    v = u[:, 0]
    r = v * (1.0 - (1.0 - u[:, 1]) ** (1.0 / beta))
    r[np.argmin(v)] = 0.0
    c = r / 2.0 + u[:, 2] * (v - r / 2.0)
    lo, hi = c - r / 2.0, c + r / 2.0
    rows = []
    for i in range(n):
        prey = np.nonzero((v >= lo[i]) & (v <= hi[i]) & (r[i] > 0))[0]
        rows.append(prey.astype(np.uint32))
    prey_ptr = np.zeros(n + 1, dtype=np.uint32)
    prey_ptr[1:] = np.cumsum([x.size for x in rows])
    prey_idx = np.concatenate(rows).astype(np.uint32) if n else np.zeros(0, np.uint32)
    return prey_ptr, prey_idx


def graph_from_csr(n: int, row_ptr, col, name: str = "") -> Graph:
    """A Graph from a simple undirected CSR (sorted rows), e.g. a niche overlap graph."""
    return Graph(n, np.asarray(row_ptr, dtype=np.uint32), np.asarray(col, dtype=np.uint32), name)


# ---------------------------------------------------------------- packing helpers

def pack(graphs: Sequence[Graph]):
    """Concatenate CSRs for a batch call: returns (n[], row_off[], row_ptr_all, col_off[], col_all).

    ``row_off[g]`` indexes ``row_ptr_all`` (each graph contributes n_g + 1 entries) and
    ``col_off[g]`` indexes ``col_all``; both have count + 1 entries."""
    ns = np.array([g.n for g in graphs], dtype=np.uint32)
    row_off = np.zeros(len(graphs) + 1, dtype=np.uint64)
    col_off = np.zeros(len(graphs) + 1, dtype=np.uint64)
    row_off[1:] = np.cumsum([g.n + 1 for g in graphs])
    col_off[1:] = np.cumsum([g.col.size for g in graphs])
    rp = np.concatenate([g.row_ptr for g in graphs]).astype(np.uint32) if graphs else np.zeros(0, np.uint32)
    cl = np.concatenate([g.col for g in graphs]).astype(np.uint32) if graphs else np.zeros(0, np.uint32)
    return ns, row_off, rp, col_off, cl
