/*
 * CPU ORACLE for chordless-cycle enumeration (arXiv 1410.4876).  TEST INFRASTRUCTURE ONLY:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg may load this
 * library.  It shares no code with the CUDA path.
 *
 * Plain, slow and written to be checked against the paper by eye:
 *   cco_degree_labeling  - degree labelling, Section 2 (definition of G_1, G_{i+1} = G_i - u_i,
 *                          l(u_i) = i).  The paper does not say which minimum-degree vertex
 *                          to take when several tie; this oracle takes the smallest vertex id.
 *   cco_enumerate        - Algorithm 1 (SequentialChordlessCycles): triplet set T(G) and
 *                          triangles, then the worklist loop with the label test, the chord
 *                          test against v_2..v_{t-1} and the close test against v_1.
 *                          T is processed as a LIFO stack (the paper leaves the order open).
 *   cco_bruteforce       - the definition itself (Section 1): every vertex subset S, |S| >= 3,
 *                          whose induced subgraph is connected with every degree equal to 2.
 *   cco_niche_overlap    - the niche overlap graph of a food web (Section 5, after Wilson and
 *                          Watkins): distinct species x, y are adjacent when some species z is
 *                          a prey of both (arcs x -> z and y -> z).
 *
 * Lengths count vertices.  max_len bounds the cycle length (0 = no bound); a path of t
 * vertices is kept for expansion only while t < L' = min(max_len, n).
 *
 * Cycle hash (order independent, exact): r(v) = mix((v + 1) * GAMMA),
 * h(C) = mix(sum_{v in C} r(v) + |C| * GAMMA), H = sum_C h(C), all modulo 2^64, where mix
 * is the SplitMix64 output finaliser (Steele, Lea, Flood 2014; constants of Vigna's
 * public-domain splitmix64.c) and v are the caller's vertex ids.
 *
 * Canonical ordered form of a cycle (for cycle lists): start at its smallest vertex id
 * and continue towards the smaller of that vertex's two cycle neighbours.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t cco_vertex_hash(uint32_t v) { return mix((uint64_t)(v + 1ULL) * GAMMA); }

uint64_t cco_cycle_hash(const uint32_t* c, uint32_t k) {
  uint64_t s = 0;
  for (uint32_t i = 0; i < k; ++i) s += cco_vertex_hash(c[i]);
  return mix(s + (uint64_t)k * GAMMA);
}

uint64_t cco_splitmix64_next(uint64_t* state) {
  *state += GAMMA;
  return mix(*state);
}

/* ------------------------------------------------------------------ graph access */

/* Adjacency test by binary search in the sorted neighbour row of x (the compact
 * representation of Section 4.2 keeps rows sorted for exactly this). */
static int adjacent(const uint32_t* row_ptr, const uint32_t* col, uint32_t x, uint32_t y) {
  uint32_t lo = row_ptr[x], hi = row_ptr[x + 1];
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo) / 2;
    if (col[mid] == y) return 1;
    if (col[mid] < y) lo = mid + 1; else hi = mid;
  }
  return 0;
}

/* ------------------------------------------------------------------ degree labelling */

/* Section 2: G_1 = G; at step i pick u_i of minimum degree in G_i (ties: smallest id),
 * set l(u_i) = i and remove it.  label[] receives 1..n.  O(n^2 + m). */
void cco_degree_labeling(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t* label) {
  int64_t* deg = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  char* removed = (char*)calloc(n ? n : 1, 1);
  for (uint32_t v = 0; v < n; ++v) deg[v] = (int64_t)(row_ptr[v + 1] - row_ptr[v]);
  for (uint32_t i = 1; i <= n; ++i) {
    uint32_t u = n;
    for (uint32_t v = 0; v < n; ++v)
      if (!removed[v] && (u == n || deg[v] < deg[u])) u = v;
    label[u] = i;
    removed[u] = 1;
    for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
      if (!removed[col[e]]) deg[col[e]] -= 1;
  }
  free(deg);
  free(removed);
}

/* ------------------------------------------------------------------ output helpers */

typedef struct {
  uint64_t* hist;       /* [L'+1], hist[k] = chordless cycles with k vertices        */
  uint64_t hash;
  uint32_t* cyc_vertices; /* optional canonical cycle list                          */
  uint64_t* cyc_offsets;  /* [cap_cycles + 1]                                       */
  uint64_t cap_cycles, cap_vertices;
  uint64_t n_cycles, n_vertices; /* required sizes (may exceed the capacities)      */
} sink_t;

static void canonical_order(const uint32_t* c, uint32_t k, uint32_t* out) {
  uint32_t i0 = 0;
  for (uint32_t i = 1; i < k; ++i) if (c[i] < c[i0]) i0 = i;
  uint32_t nxt = c[(i0 + 1) % k], prv = c[(i0 + k - 1) % k];
  int dir = (nxt < prv) ? 1 : -1;
  for (uint32_t j = 0; j < k; ++j) out[j] = c[(i0 + (uint32_t)((int64_t)k + dir * (int64_t)j) % k) % k];
}

static void emit_cycle(sink_t* s, const uint32_t* c, uint32_t k) {
  s->hist[k] += 1;
  s->hash += cco_cycle_hash(c, k);
  if (s->cyc_offsets) {
    if (s->n_cycles < s->cap_cycles && s->n_vertices + k <= s->cap_vertices) {
      canonical_order(c, k, s->cyc_vertices + s->n_vertices);
      s->cyc_offsets[s->n_cycles] = s->n_vertices;
      s->cyc_offsets[s->n_cycles + 1] = s->n_vertices + k;
    }
  }
  s->n_cycles += 1;
  s->n_vertices += k;
}

/* ------------------------------------------------------------------ Algorithm 1 */

typedef struct { uint32_t* v; uint64_t used, cap; } pool_t;

static int pool_reserve(pool_t* p, uint64_t extra) {
  if (p->used + extra <= p->cap) return 0;
  uint64_t nc = p->cap ? p->cap : 1024;
  while (nc < p->used + extra) nc *= 2;
  uint32_t* nv = (uint32_t*)realloc(p->v, nc * sizeof(uint32_t));
  if (!nv) return -1;
  p->v = nv; p->cap = nc;
  return 0;
}

/*
 * Algorithm 1.  Returns 0, or -1 on allocation failure.
 *   hist[0..L']       out: per-length cycle counts (caller zeroes nothing; we zero it)
 *   tcount[0..L']     out (optional): tcount[t] = number of paths of t vertices placed in T
 *   part, nparts      process only the initial triplets and triangles <x,u,y> of this
 *                     part: mix((u * n + x) * n + y) mod nparts == part, original ids (the
 *                     library's split of T(G); every triplet roots its own subtree, Section
 *                     4.3, so the parts add up to the whole); nparts = 1 runs everything.
 */
/* The part of the initial triplet or triangle <x,u,y>: mix((u n + x) n + y) mod nparts. */
static int in_part(uint32_t x, uint32_t u, uint32_t y, uint32_t n, uint32_t part, uint32_t nparts) {
  if (nparts <= 1) return 1;
  uint64_t key = ((uint64_t)u * n + x) * n + y;
  return mix(key) % nparts == part;
}

int cco_enumerate(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t max_len,
                  uint32_t part, uint32_t nparts,
                  uint64_t* hist, uint64_t* hash, uint64_t* tcount,
                  uint32_t* cyc_vertices, uint64_t* cyc_offsets, uint64_t cap_cycles,
                  uint64_t cap_vertices, uint64_t* n_cycles, uint64_t* n_vertices) {
  uint32_t L = (max_len == 0 || max_len > n) ? n : max_len;
  memset(hist, 0, sizeof(uint64_t) * (L + 1));
  if (tcount) memset(tcount, 0, sizeof(uint64_t) * (L + 1));
  sink_t s = {hist, 0, cyc_vertices, cyc_offsets, cap_cycles, cap_vertices, 0, 0};
  if (cyc_offsets && cap_cycles > 0) cyc_offsets[0] = 0;
  if (nparts == 0) nparts = 1;

  uint32_t* label = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  /* Algorithm 1 begins with the degree labelling */
  cco_degree_labeling(n, row_ptr, col, label);

  /* T is a LIFO stack of paths; path j occupies pool.v[off[j] .. off[j] + len[j]). */
  pool_t pool = {0, 0, 0};
  uint64_t *off = NULL, *len = NULL;
  uint64_t top = 0, cap = 0;
  uint32_t* p = NULL; /* the path taken from T, copied out of the pool */
  uint64_t pcap = 0;
  int rc = 0;
#define PUSH_PATH(src, t_, extra)                                                        \
  do {                                                                                   \
    if (top == cap) {                                                                    \
      cap = cap ? cap * 2 : 1024;                                                        \
      off = (uint64_t*)realloc(off, cap * sizeof(uint64_t));                             \
      len = (uint64_t*)realloc(len, cap * sizeof(uint64_t));                             \
      if (!off || !len) { rc = -1; goto done; }                                          \
    }                                                                                    \
    if (pool_reserve(&pool, (t_) + 1)) { rc = -1; goto done; }                           \
    memcpy(pool.v + pool.used, (src), sizeof(uint32_t) * ((t_) - 1));                   \
    pool.v[pool.used + (t_) - 1] = (extra);                                              \
    off[top] = pool.used; len[top] = (t_); pool.used += (t_); top += 1;                  \
    if (tcount) tcount[(t_)] += 1;                                                       \
  } while (0)

  if (L >= 3) {
    /* Algorithm 1, initial sets: triplets <x,u,y> with x,y in Adj(u) and l(u) < l(x) < l(y);
     * (x,y) in E gives a triangle (cycle), otherwise an initial chordless path. */
    for (uint32_t u = 0; u < n; ++u)
      for (uint32_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a)
        for (uint32_t b = row_ptr[u]; b < row_ptr[u + 1]; ++b) {
          uint32_t x = col[a], y = col[b];
          if (!(label[u] < label[x] && label[x] < label[y])) continue;
          if (!in_part(x, u, y, n, part, nparts)) continue;
          uint32_t c[3] = {x, u, y};
          if (adjacent(row_ptr, col, x, y)) {
            emit_cycle(&s, c, 3);
          } else if (L > 3) {
            PUSH_PATH(c, 3, y);
          }
        }
  }

  /* Algorithm 1, main loop: while T is not empty take a path p = <v_1..v_t> and try every
   * neighbour v of v_t. */
  while (top > 0) {
    top -= 1;
    uint64_t t = len[top];
    if (pcap < t + 1) { pcap = 2 * (t + 1); p = (uint32_t*)realloc(p, pcap * sizeof(uint32_t)); if (!p) { rc = -1; goto done; } }
    memcpy(p, pool.v + off[top], t * sizeof(uint32_t));
    pool.used = off[top]; /* stack discipline: this path was the last one pushed */
    uint32_t v1 = p[0], v2 = p[1], vt = p[t - 1];
    for (uint32_t e = row_ptr[vt]; e < row_ptr[vt + 1]; ++e) {
      uint32_t v = col[e];
      /* label test against v_2 and chord test against v_2..v_{t-1};
       * v not on p is implied by those tests and is checked explicitly as well. */
      if (!(label[v] > label[v2])) continue;
      int on_path = 0, chord = 0;
      for (uint64_t i = 0; i < t; ++i) if (p[i] == v) on_path = 1;
      if (on_path) continue;
      for (uint64_t i = 1; i + 1 < t; ++i)
        if (adjacent(row_ptr, col, v, p[i])) { chord = 1; break; }
      if (chord) continue;
      if (adjacent(row_ptr, col, v, v1)) {
        /* v adjacent to v_1: <p, v> is a chordless cycle of t + 1 vertices */
        if (t + 1 <= L) { p[t] = v; emit_cycle(&s, p, (uint32_t)(t + 1)); }
      } else if (t + 1 < L) {
        /* otherwise <p, v> is a chordless path kept for expansion */
        PUSH_PATH(p, (uint32_t)(t + 1), v);
      }
    }
  }
done:
#undef PUSH_PATH
  *hash = s.hash;
  if (n_cycles) *n_cycles = s.n_cycles;
  if (n_vertices) *n_vertices = s.n_vertices;
  free(p); free(off); free(len); free(pool.v); free(label);
  return rc;
}

/* ------------------------------------------------------------------ brute force */

/* The definition (Section 1): S with |S| >= 3 induces a chordless cycle iff every vertex
 * of S has exactly two neighbours in S and G[S] is connected.  n <= 30.  Returns 0, or
 * -1 if n is too large. */
int cco_bruteforce(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t max_len,
                   uint64_t* hist, uint64_t* hash,
                   uint32_t* cyc_vertices, uint64_t* cyc_offsets, uint64_t cap_cycles,
                   uint64_t cap_vertices, uint64_t* n_cycles, uint64_t* n_vertices) {
  if (n > 30) return -1;
  uint32_t L = (max_len == 0 || max_len > n) ? n : max_len;
  memset(hist, 0, sizeof(uint64_t) * (L + 1));
  sink_t s = {hist, 0, cyc_vertices, cyc_offsets, cap_cycles, cap_vertices, 0, 0};
  if (cyc_offsets && cap_cycles > 0) cyc_offsets[0] = 0;
  uint32_t adjm[32];
  for (uint32_t v = 0; v < n; ++v) {
    adjm[v] = 0;
    for (uint32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) adjm[v] |= 1u << col[e];
  }
  uint32_t c[32];
  for (uint64_t S = 1; S < (1ULL << n); ++S) {
    uint32_t k = (uint32_t)__builtin_popcountll(S);
    if (k < 3 || k > L) continue;
    int ok = 1;
    for (uint32_t v = 0; v < n && ok; ++v)
      if ((S >> v) & 1) ok = (__builtin_popcount(adjm[v] & (uint32_t)S) == 2);
    if (!ok) continue;
    /* connected: walk the 2-regular induced subgraph from its smallest vertex */
    uint32_t start = (uint32_t)__builtin_ctzll(S), prev = start, cur = start, steps = 0;
    uint32_t nb = adjm[start] & (uint32_t)S;
    uint32_t a = (uint32_t)__builtin_ctz(nb), b = 31 - (uint32_t)__builtin_clz(nb);
    c[0] = start;
    cur = (a < b) ? a : b; /* towards the smaller neighbour */
    steps = 1;
    while (cur != start && steps <= k) {
      c[steps++] = cur;
      uint32_t nx = adjm[cur] & (uint32_t)S & ~(1u << prev);
      prev = cur;
      cur = (uint32_t)__builtin_ctz(nx);
    }
    if (cur != start || steps != k) continue; /* more than one component */
    emit_cycle(&s, c, k);
  }
  *hash = s.hash;
  if (n_cycles) *n_cycles = s.n_cycles;
  if (n_vertices) *n_vertices = s.n_vertices;
  return 0;
}

/* Triplet set size |T(G)| (Section 2) for the degree labelling, by its definition. */
uint64_t cco_triplet_count(uint32_t n, const uint32_t* row_ptr, const uint32_t* col) {
  uint32_t* label = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  cco_degree_labeling(n, row_ptr, col, label);
  uint64_t cnt = 0;
  for (uint32_t u = 0; u < n; ++u)
    for (uint32_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a)
      for (uint32_t b = row_ptr[u]; b < row_ptr[u + 1]; ++b) {
        uint32_t x = col[a], y = col[b];
        if (label[u] < label[x] && label[x] < label[y] && !adjacent(row_ptr, col, x, y)) cnt++;
      }
  free(label);
  return cnt;
}

/* ------------------------------------------------------------------ niche overlap graph */

/* Section 5: the food webs are turned into niche overlap graphs.  prey_idx[prey_ptr[x] ..
 * prey_ptr[x+1]) lists the prey of x (arcs x -> z).  x != y are adjacent iff they share a
 * prey.  Writes the CSR with ascending rows; out_col needs room for n (n - 1) ids.
 * Returns row_ptr[n]. */
uint64_t cco_niche_overlap(uint32_t n, const uint32_t* prey_ptr, const uint32_t* prey_idx, uint32_t* out_row_ptr,
                           uint32_t* out_col) {
  uint64_t nnz = 0;
  for (uint32_t x = 0; x < n; ++x) {
    out_row_ptr[x] = (uint32_t)nnz;
    for (uint32_t y = 0; y < n; ++y) {
      if (y == x) continue;
      int share = 0;
      for (uint32_t a = prey_ptr[x]; a < prey_ptr[x + 1] && !share; ++a)
        for (uint32_t b = prey_ptr[y]; b < prey_ptr[y + 1]; ++b)
          if (prey_idx[a] == prey_idx[b]) { share = 1; break; }
      if (share) out_col[nnz++] = y;
    }
  }
  out_row_ptr[n] = (uint32_t)nnz;
  return nnz;
}
