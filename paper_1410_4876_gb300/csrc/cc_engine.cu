// Persistent expansion engine: Algorithm 3 (ExpandingChordlessPathsParallel) executed
// level after level inside ONE cooperative launch, replacing the host relaunch loop of
// Algorithm 4 by grid-wide barriers (Section 4.4 uses persistent threads within a level;
// here the persistence also spans the levels).
//
// Control.  Every block keeps an identical copy of the frame chain's top in shared
// memory and applies the same deterministic plan/commit rules, so the only grid-wide
// communication per step is the child counters read after the barrier.  Block 0 also
// mirrors frames into global memory so any block can pop back to them.
//
// Per step: take the top frame, choose how much of it to expand (all of it if the exact
// or bounded child count fits the free arena, else the largest chunk that fits; that
// chunk's subtree then runs depth-first; a bitset level whose children are known exactly
// and grow slowly, or any such level of a sparse graph, is expanded together with them;
// with a streamed cycle list, no more than the list's room can take), expand those
// paths, list their children as (path, vertex) entries worked off one per lane, give each
// warp's child list its slots with one atomic, accumulate cycles.
//
// Expansion forms: process_bitset_flat / process_bitset_fused (one graph, bitset
// adjacency), process_multi_flat (batch and serving), process_bitset /
// process_bitset_fused_lane (the small-level cluster phase), process_csr_coop /
// process_csr_last / process_csr_long_warp (CSR adjacency).
#include <cooperative_groups.h>
#include <cstddef>
#include <mutex>
#include <utility>
#include <vector>

#include "cc_internal.cuh"

namespace cc {

constexpr int kMaxThreads = 256;    // persistent grid blocks
constexpr int kSmallThreads = 1024; // small-phase cluster blocks

struct StepPlan {
  unsigned long long src_base, src_stride, begin, end;
  unsigned long long dst_base, dst_stride;
  unsigned long long s;
  unsigned int t;
  unsigned int done;
  unsigned int fuse;  // 1: expand levels t and t+1 in this step, store level t+2
  unsigned int pad_;
};

struct LocalState {
  Frame cur;
  Frame child;
  unsigned long long bot, top, chunk, peak;
  unsigned int depth, has_child, gen, fused;
  unsigned long long expanded;  // paths expanded by the planned step (both levels of a fused one)
};

// (word by word, bypassing L1: another block may have stored the frame)
static_assert(offsetof(Frame, next) == 40 && offsetof(Frame, ncl) == 48 && offsetof(Frame, t) == 56 &&
                  offsetof(Frame, end) == 60 && sizeof(Frame) == 64,
              "load_frame reads the Frame layout word by word");
__device__ __forceinline__ Frame load_frame(const Frame* f) {
  Frame r;
  const unsigned long long* q = reinterpret_cast<const unsigned long long*>(f);
  r.base = __ldcg(q + 0);
  r.bytes = __ldcg(q + 1);
  r.stride = __ldcg(q + 2);
  r.count = __ldcg(q + 3);
  r.cursor = __ldcg(q + 4);
  r.next = __ldcg(q + 5);
  r.ncl = __ldcg(q + 6);
  const unsigned long long te = __ldcg(q + 7);
  r.t = (unsigned int)(te & 0xFFFFFFFFull);
  r.end = (unsigned int)(te >> 32);
  return r;
}
__device__ __forceinline__ void store_frame(Frame* f, const Frame& r) { *f = r; }

template <Kind K>
struct KindTraits {
  static constexpr int W = K == Kind::Bitset2 ? 2 : (K == Kind::Bitset4 ? 4 : 1);
  static constexpr bool multi = K == Kind::Multi;
  static constexpr bool csr = is_csr(K);
  static constexpr int cap = K == Kind::Csr16 ? 16 : (K == Kind::Csr32 ? 32 : 64);
  // paths per thread per tile, and the minimum resident 256-thread blocks per SM the
  // register allocation must allow (4 blocks = 64 registers per thread, 3 = 85, 2 = 128)
  static constexpr int P = K == Kind::Bitset4 ? 1 : (K == Kind::Bitset1 ? 3 : 2);
  static constexpr int minB =
      (K == Kind::Csr || K == Kind::Csr32) ? 2 : ((K == Kind::Csr16 || K == Kind::Bitset1) ? 3 : 4);
  // paths per thread per round of the flattened single-graph form (one slot atomic per
  // warp per round)
  static constexpr int PF = K == Kind::Bitset1 ? 3 : (K == Kind::Bitset2 ? 2 : 1);
  // children staged per batch in a two-level step, in rounds of 32 (shared memory bound)
  static constexpr int PF2 = K == Kind::Bitset1 ? 2 : 1;
};

template <Kind K>
__device__ __forceinline__ unsigned long long region_bytes(unsigned long long stride, unsigned int t_child) {
  if constexpr (KindTraits<K>::csr) return csr_region_bytes(stride, t_child);
  else if constexpr (KindTraits<K>::multi) return multi_region_bytes(stride);
  else return bitset_region_bytes(stride, KindTraits<K>::W);
}
template <Kind K>
__device__ __forceinline__ unsigned long long record_bytes(unsigned int t_child) {
  if constexpr (KindTraits<K>::csr) return 2ull * csr_rec_u16(t_child);
  else if constexpr (KindTraits<K>::multi) return 21ull;
  else return 8ull * KindTraits<K>::W + 12ull;
}

// ------------------------------------------------------------------ control (thread 0)

// In sparse graphs (at most this many children per path) two-level steps are taken
// however fast the levels grow: the per-step floor (barrier and counter round trips) and
// the frontier traffic of the skipped level outweigh the staging cost.
constexpr unsigned int kFuseSparseMaxch = 4;
// The cluster phase's two-level form (one path per lane) is used up to this many bitset
// words (wider rows would spill registers at 1024 threads per block).
constexpr int kFuseLaneMaxW = 1;

template <Kind K>
__device__ bool plan_step(const EngineParams& p, LocalState& st, StepPlan& pl) {
  while (st.depth > 0 && st.cur.cursor >= st.cur.count) {  // pop finished frames
    if (st.cur.end == 0) st.bot = st.cur.base; else st.top = st.cur.base + st.cur.bytes;
    st.depth -= 1;
    if (st.depth > 0) st.cur = load_frame(&p.frames[st.depth - 1]);
  }
  if (st.depth == 0) return false;
  const Frame& f = st.cur;
  const unsigned long long rem = f.count - f.cursor;
  const unsigned int t = f.t;
  unsigned long long need, lim = rem;
  if constexpr (KindTraits<K>::csr) {
    if (p.cyc_stream && t + 1 <= p.L) {
      // streamed cycle list: the step's closings (t+1 vertices each) must fit the list's
      // room, or the step stops here and the host drains the list and resumes (the list
      // counters are final after the barrier).  A whole frame with a known closing bound
      // is taken if the bound fits, and waits for an empty list if only that would hold
      // it; otherwise a path closes at most maxch cycles and the step takes no more paths
      // than the room holds at that rate.
      const unsigned long long uc = ld_relaxed_u64(&p.ctl->cyc_count), uv = ld_relaxed_u64(&p.ctl->cyc_verts);
      const unsigned long long roomc = uc < p.cyc_cap_c ? p.cyc_cap_c - uc : 0ull;
      const unsigned long long roomv = uv < p.cyc_cap_v ? p.cyc_cap_v - uv : 0ull;
      const bool whole = f.cursor == 0 && f.ncl != kNoNext;
      if (whole && f.ncl <= roomc && f.ncl * (t + 1) <= roomv) {
        lim = rem;
      } else if (whole && (uc || uv) && f.ncl <= p.cyc_cap_c && f.ncl * (t + 1) <= p.cyc_cap_v) {
        return false;
      } else {
        lim = min(lim, min(roomc / p.maxch, roomv / ((unsigned long long)p.maxch * (t + 1))));
        if (lim == 0) return false;
      }
    }
    // CSR frames carry an upper bound on their children (sum of deg(v_t) - 1)
    need = (t + 1 < p.L) ? ((f.cursor == 0 && f.next != kNoNext && lim == rem) ? f.next : lim * p.maxch) : 0ull;
  } else if constexpr (KindTraits<K>::multi) {
    need = (f.cursor == 0 && f.next != kNoNext) ? f.next : rem * p.maxch;
  } else {
    need = (t + 1 >= p.L) ? 0ull : ((f.cursor == 0 && f.next != kNoNext) ? f.next : rem * p.maxch);
  }
  const unsigned long long res = KindTraits<K>::multi ? p.reserve : 0ull;
  unsigned long long cap = need + (need || res ? res : 0ull);
  st.chunk = lim;
  st.has_child = 0;
  st.fused = 0;
  pl.fuse = 0;
  if constexpr (!KindTraits<K>::multi && !KindTraits<K>::csr) {
    // Two levels in one step: a whole frame whose children (level t+1) are known exactly
    // is expanded, its children are expanded in the same step without being stored, and
    // only the grandchildren (level t+2) are stored.  Their count is bounded by
    // children * maxch; the step is taken only when that bound fits the free arena
    // (otherwise the level runs alone and may be split into depth-first chunks), and,
    // unless the graph is sparse, only while the frontier grows by at most 1.3x per level
    // (measured: in denser graphs, steps of fast-growing levels are quicker one level at a
    // time).
    if (p.fuse_ok && (!p.cluster || (KindTraits<K>::W <= kFuseLaneMaxW && f.next <= p.handover)) && t + 1 < p.L &&
        f.cursor == 0 && f.next != kNoNext && f.next > 0 &&
        (f.next * 10ull <= f.count * 13ull || p.maxch <= kFuseSparseMaxch)) {
      const unsigned long long need2 = (t + 2 < p.L) ? f.next * p.maxch : 0ull;
      const unsigned long long rb2 = record_bytes<K>(t + 2);
      const unsigned long long freeb = st.top - st.bot;
      // (a multiply-compare: the planner runs on one thread per block every step)
      if (freeb > 1024 && (round_up(need2, 8) + 8) * rb2 <= freeb - 1024) {
        st.fused = 1;
        pl.fuse = 1;
        if (need2 > 0) {
          const unsigned long long stride = round_up(need2, 8);
          const unsigned long long bytes = region_bytes<K>(stride, t + 2);
          Frame& c = st.child;
          c.end = 1u - f.end;
          c.base = c.end ? st.top - bytes : st.bot;
          c.bytes = bytes;
          c.stride = stride;
          c.count = 0;
          c.cursor = 0;
          c.next = kNoNext;
          c.ncl = kNoNext;
          c.t = t + 2;
          st.has_child = 1;
          st.peak = max(st.peak, p.arena_bytes - (freeb - bytes));
        }
        cap = 0;  // the single-level plan below is not used
      }
    }
  }
  if (cap > 0) {
    const unsigned long long rb = record_bytes<K>(t + 1);
    const unsigned long long freeb = st.top - st.bot;
    // the division is only needed when the level does not fit (the common case is a
    // multiply-compare)
    const bool fits = freeb > 1024 && (round_up(cap, 8) + 8) * rb <= freeb - 1024;
    unsigned long long maxcap = fits ? cap : (freeb > 1024 ? ((freeb - 1024) / rb) & ~7ull : 0ull);
    // (bitset and batch frames hold fewer than 2^32 records: their forms index them with 32
    // bits)
    if constexpr (!KindTraits<K>::csr) maxcap = min(maxcap, 0xFFFF0000ull);
    if (cap > maxcap) {
      // Spill: this chunk's subtree runs depth-first before the rest of the frame, and
      // each deeper stored level of that subtree needs room too, so the chunk's children
      // get only an equal share of the free space among those levels.
      const unsigned long long levels =
          KindTraits<K>::multi ? (st.depth + 4 < p.L ? p.L - 3ull - st.depth : 1ull)
                               : (p.L > t + 2 ? (unsigned long long)(p.L - t - 1) : 1ull);
      const unsigned long long share = maxcap / levels;
      unsigned long long ch = share > res ? (share - res) / p.maxch : 0ull;
      if (ch == 0 && maxcap >= res + p.maxch) ch = 1;
      // host frontier: rather than expanding this level in small chunks (or failing), stop
      // so that the host moves the frames below to host memory and resumes with the arena
      // free (the state written back at kernel end is this step's, unchanged)
      if (p.offload_min && st.depth >= 2 && ch < p.offload_min) {
        if (blockIdx.x == 0) p.ctl->want_offload = 1u;
        return false;
      }
      if (ch == 0) {
        set_err(p.ctl, kDevCapacity, (int)t);
        return false;
      }
      if (ch < st.chunk) {
        st.chunk = ch;
        if (blockIdx.x == 0) p.ctl->spilled = 1;
      }
      cap = st.chunk * p.maxch + res;
    }
    const unsigned long long stride = round_up(cap, 8);
    const unsigned long long bytes = region_bytes<K>(stride, t + 1);
    Frame& c = st.child;
    c.end = 1u - f.end;
    c.base = c.end ? st.top - bytes : st.bot;
    c.bytes = bytes;
    c.stride = stride;
    c.count = 0;
    c.cursor = 0;
    c.next = kNoNext;
    c.ncl = kNoNext;
    c.t = KindTraits<K>::multi ? 0u : t + 1;
    st.has_child = 1;
    st.peak = max(st.peak, p.arena_bytes - (freeb - bytes));
  }
  st.expanded = st.chunk + (st.fused ? f.next : 0ull);
  pl.src_base = f.base;
  pl.src_stride = f.stride;
  pl.begin = f.cursor;
  pl.end = f.cursor + st.chunk;
  pl.dst_base = st.has_child ? st.child.base : 0ull;
  pl.dst_stride = st.has_child ? st.child.stride : 0ull;
  pl.t = t;
  return true;
}

template <Kind K>
__device__ void commit_step(const EngineParams& p, LocalState& st, unsigned long long c, unsigned long long nx,
                            unsigned long long ncl, bool writer) {
  const unsigned int t = st.cur.t;
  // a two-level step: its children were counted exactly before the step (the frame's next)
  if (st.fused && writer) atomicAdd(&p.tcount[t + 1], st.cur.next);
  st.cur.cursor += st.chunk;
  const bool consumed = st.cur.cursor >= st.cur.count;
  if (consumed) {
    if (st.cur.end == 0) st.bot = st.cur.base; else st.top = st.cur.base + st.cur.bytes;
    st.depth -= 1;
  } else if (writer) {
    store_frame(&p.frames[st.depth - 1], st.cur);
  }
  if (st.has_child && c > 0) {
    Frame g = st.child;
    if (c > g.stride) {  // more children than the planned bound (the writes past it were skipped)
      set_err(p.ctl, kDevCapacity, (int)t);
      c = g.stride;
    }
    g.count = c;
    g.cursor = 0;
    g.next = nx;  // exact (bitset, batch) or an upper bound (CSR)
    g.ncl = ncl;
    if (g.end) st.top = g.base; else st.bot = g.base + g.bytes;
    if (st.depth >= p.max_depth) {
      set_err(p.ctl, kDevDepth, (int)st.depth);
      return;
    }
    if (writer) {
      store_frame(&p.frames[st.depth], g);
      if constexpr (!KindTraits<K>::multi) atomicAdd(&p.tcount[g.t], c);
    }
    st.depth += 1;
    st.cur = g;
  } else if (consumed && st.depth > 0) {
    st.cur = load_frame(&p.frames[st.depth - 1]);
  }
}

// ------------------------------------------------------------------ bitset expansion

// Batch-mode statistics of one (slot, length) key, accumulated per lane; flush() is
// warp-collective and adds the warp's sums to the slot's histogram, hash, stored-path
// count and in-flight count with one lane's atomics.
struct StatRun {
  unsigned int key;
  unsigned int c = 0, k = 0, n = 0;
  unsigned long long h = 0;
  __device__ __forceinline__ void add(unsigned int cc, unsigned int kk, unsigned long long hh) {
    c += cc;
    k += kk;
    n += 1;
    h += hh;
  }
  __device__ __forceinline__ void flush(const EngineParams& p, unsigned long long s) {
    const unsigned int sc = __reduce_add_sync(0xffffffffu, c);
    const unsigned int sk = __reduce_add_sync(0xffffffffu, k);
    const unsigned int sn = __reduce_add_sync(0xffffffffu, n);
    const unsigned long long sh = warp_sum_u64(h);
    if ((threadIdx.x & 31) == 0 && key != 0xFFFFFFFFu && sn) {
      const unsigned int g = key >> 6, tt = key & 63u;
      const unsigned long long hb = (unsigned long long)g * kMultiHistStride;
      if (sc) atomicAdd(&p.hist[hb + tt + 1], (unsigned long long)sc);
      if (sh) atomicAdd(&p.hash[g], sh);
      if (sk) atomicAdd(&p.tcount[hb + tt + 1], (unsigned long long)sk);
      if (p.live)
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.live[g]),
                  (unsigned long long)((long long)sk - (long long)sn));
      if (p.last_step && sn) atomicMax(&p.last_step[g], (unsigned int)s + 1u);
    }
    c = k = n = 0;
    h = 0;
  }
};

// Algorithm 3 on bitset records.  For a path p = <v1 .. vt> with blocked set B:
//   cand  = Adj(vt) & ~B      label test (l(v) > l(v2)), v not on p, chord test v2..v_{t-1}
//   close = cand & Adj(v1)    chordless cycles <p, v> of t+1 vertices
//   child = cand & ~Adj(v1)   chordless paths <p, v>, blocked set B | Adj(vt)
// The exact child count of each new path is popc(Adj(v) & ~(B | Adj(vt)) & ~Adj(v1)),
// summed so the next frame's size is known before it is expanded.
template <Kind K>
__device__ __forceinline__ void process_bitset(const EngineParams& p, const StepPlan& pl,
                                               const unsigned long long* adj, const unsigned long long* rtab,
                                               unsigned int* s_warp, unsigned long long* s_red,
                                               unsigned long long* s_base, unsigned long long* cntp,
                                               unsigned long long* nxtp) {
  constexpr int W = KindTraits<K>::W;
  constexpr int P = KindTraits<K>::P;
  static_assert(!KindTraits<K>::multi, "batch records are expanded by process_multi_flat");
  const unsigned int tid = threadIdx.x;
  const unsigned long long ss = pl.src_stride, ds = pl.dst_stride;
  const unsigned long long* sB = reinterpret_cast<const unsigned long long*>(p.arena + pl.src_base);
  const unsigned long long* sH = sB + W * ss;
  const unsigned int* sM = reinterpret_cast<const unsigned int*>(sH + ss);
  unsigned long long* dB = reinterpret_cast<unsigned long long*>(p.arena + pl.dst_base);
  unsigned long long* dH = dB + W * ds;
  unsigned int* dM = reinterpret_cast<unsigned int*>(dH + ds);
  const bool store = ds != 0;
  const unsigned int t = pl.t, L = p.L;
  const unsigned long long s = pl.s;
  const bool close_ok = t + 1 <= L, next_ok = t + 2 < L;
  unsigned long long nx = 0, ncyc = 0, hacc = 0;

  // thread-interleaved grid stride: path i0 + j*T (j < P) for thread gtid, T threads in
  // the grid, so the last round of a step is spread over every thread (no block tiles)
  const unsigned long long T = (unsigned long long)gridDim.x * blockDim.x;
  // warp w of block b takes the (w * gridDim + b)-th group of 32 paths, so the warps of a
  // small step land on different SMs
  const unsigned long long gwarp = ((unsigned long long)(tid >> 5) * gridDim.x + blockIdx.x) * 32ull;
  // the bound is tested on the warp's first thread so every lane runs the same iterations
  // (the body uses full-warp collectives)
  // pf <= P paths per thread per round (a runtime knob; rounds j >= pf are empty)
  const unsigned int pf = p.pf >= 1 && p.pf <= (unsigned)P ? p.pf : (unsigned)P;
  for (unsigned long long wb = pl.begin + gwarp; wb < pl.end; wb += pf * T) {
    const unsigned long long t0 = wb + (tid & 31);
    unsigned long long B[P][W], H[P], ch[P][W];
    unsigned int M[P];
    unsigned int nch = 0;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const unsigned long long i = t0 + (unsigned long long)j * T;
      const bool valid = (unsigned)j < pf && i < pl.end;
#pragma unroll
      for (int k = 0; k < W; ++k) B[j][k] = valid ? ldcg64(sB + k * ss + i) : ~0ull;
      H[j] = valid ? ldcg64(sH + i) : 0ull;
      M[j] = valid ? ldcg32(sM + i) : 0u;
      const unsigned int v1 = M[j] & 0xFFFFu, vt = M[j] >> 16;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        const unsigned long long at = adj[(unsigned long long)vt * W + k];
        const unsigned long long a1 = adj[(unsigned long long)v1 * W + k];
        const unsigned long long cand = at & ~B[j][k];
        unsigned long long close = cand & a1;
        ch[j][k] = store ? (cand & ~a1) : 0ull;
        nch += __popcll(ch[j][k]);
        if (close_ok) {
          ncyc += __popcll(close);
          while (close) {
            const unsigned int v = 64u * k + __ffsll((long long)close) - 1;
            close &= close - 1;
            hacc += mix64(H[j] + rtab[v] + (unsigned long long)(t + 1) * kGamma);
          }
        }
      }
    }
    if (store) {
      // children slots: warp scan and one atomic per warp (no block barrier)
      const unsigned long long off = warp_slots(nch, &cntp[s % 3]);
      if (__any_sync(0xffffffffu, nch != 0)) {
        unsigned long long slot = off;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          unsigned long long any = 0;
#pragma unroll
          for (int k = 0; k < W; ++k) any |= ch[j][k];
          if (!any) continue;
          const unsigned int v1 = M[j] & 0xFFFFu, vt = M[j] >> 16;
          unsigned long long nb[W], a1[W];
#pragma unroll
          for (int k = 0; k < W; ++k) {
            nb[k] = B[j][k] | adj[(unsigned long long)vt * W + k];
            a1[k] = adj[(unsigned long long)v1 * W + k];
          }
#pragma unroll
          for (int k = 0; k < W; ++k) {
            unsigned long long b = ch[j][k];
            while (b) {
              const unsigned int v = 64u * k + __ffsll((long long)b) - 1;
              b &= b - 1;
              if (slot < ds) {
#pragma unroll
                for (int q = 0; q < W; ++q) dB[q * ds + slot] = nb[q];
                dH[slot] = H[j] + rtab[v];
                dM[slot] = v1 | (v << 16);
                if (next_ok) {
#pragma unroll
                  for (int q = 0; q < W; ++q) nx += __popcll(adj[(unsigned long long)v * W + q] & ~nb[q] & ~a1[q]);
                }
              } else {
                set_err(p.ctl, kDevBounds, 1);
              }
              ++slot;
            }
          }
        }
      }
    }
  }
  block_sum3_u64(nx, ncyc, hacc, s_red);
  if (tid == 0) {
    if (nx) atomicAdd(&nxtp[s % 3], nx);
    if (ncyc) atomicAdd(&p.hist[t + 1], ncyc);
    if (hacc) atomicAdd(p.hash, hacc);
  }
}

// Two levels in one step, one path per lane (the small cluster phase, single graph).
// Each lane expands its path p (closings of t+1 vertices hashed), then each child
// p' = <p, v> in place: its closings (t+2 vertices) are hashed and its children are
// counted; after one slot atomic per warp, the children are walked again and the
// grandchildren <p', w> stored with B'' = B | Adj(vt) | Adj(v), H'' = H + r(v) + r(w) and
// their exact child counts.  Level t+1 is neither stored nor read back.  The lanes'
// loops are uneven, but the levels of this phase are small and their cost is the step
// floor, which this form pays once for two levels.
template <Kind K>
__device__ __forceinline__ void process_bitset_fused_lane(const EngineParams& p, const StepPlan& pl,
                                                          const unsigned long long* adj,
                                                          const unsigned long long* rtab, unsigned long long* s_red,
                                                          unsigned long long* cntp, unsigned long long* nxtp) {
  constexpr int W = KindTraits<K>::W;
  const unsigned int tid = threadIdx.x, lane = tid & 31;
  const unsigned long long ss = pl.src_stride, ds = pl.dst_stride;
  const unsigned long long* sB = reinterpret_cast<const unsigned long long*>(p.arena + pl.src_base);
  const unsigned long long* sH = sB + W * ss;
  const unsigned int* sM = reinterpret_cast<const unsigned int*>(sH + ss);
  unsigned long long* dB = reinterpret_cast<unsigned long long*>(p.arena + pl.dst_base);
  unsigned long long* dH = dB + W * ds;
  unsigned int* dM = reinterpret_cast<unsigned int*>(dH + ds);
  const unsigned int t = pl.t, L = p.L;
  const unsigned long long s = pl.s;
  // a two-level step has t + 1 < L': the children are within the bound
  const bool close2_ok = t + 2 <= L, store2 = ds != 0, next_ok = t + 3 < L;
  const unsigned long long gam1 = (unsigned long long)(t + 1) * kGamma, gam2 = (unsigned long long)(t + 2) * kGamma;
  unsigned long long nx = 0, ncyc1 = 0, ncyc2 = 0, hacc = 0;
  const unsigned long long T = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long gwarp = ((unsigned long long)(tid >> 5) * gridDim.x + blockIdx.x) * 32ull;
  for (unsigned long long wb = pl.begin + gwarp; wb < pl.end; wb += T) {
    const unsigned long long i = wb + lane;
    const bool valid = i < pl.end;
    unsigned long long nb1[W], a1[W], ch1[W];
    const unsigned long long H = valid ? ldcg64(sH + i) : 0ull;
    const unsigned int M = valid ? ldcg32(sM + i) : 0u;
    const unsigned int v1 = M & 0xFFFFu, vt = M >> 16;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const unsigned long long B = valid ? ldcg64(sB + k * ss + i) : ~0ull;
      const unsigned long long at = adj[(unsigned long long)vt * W + k];
      a1[k] = adj[(unsigned long long)v1 * W + k];
      const unsigned long long cand = at & ~B;
      ch1[k] = cand & ~a1[k];
      nb1[k] = B | at;
      unsigned long long cb = cand & a1[k];
      while (cb) {
        const unsigned int v = 64u * k + __ffsll((long long)cb) - 1;
        cb &= cb - 1;
        ++ncyc1;
        hacc += mix64(H + rtab[v] + gam1);
      }
    }
    // the children: closings of t+2 vertices, and their children counted
    unsigned int ngc = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      unsigned long long b = ch1[k];
      while (b) {
        const unsigned int v = 64u * k + __ffsll((long long)b) - 1;
        b &= b - 1;
        const unsigned long long hv = H + rtab[v];
#pragma unroll
        for (int q = 0; q < W; ++q) {
          const unsigned long long cand2 = adj[(unsigned long long)v * W + q] & ~nb1[q];
          unsigned long long cb = close2_ok ? (cand2 & a1[q]) : 0ull;
          while (cb) {
            const unsigned int w = 64u * q + __ffsll((long long)cb) - 1;
            cb &= cb - 1;
            ++ncyc2;
            hacc += mix64(hv + rtab[w] + gam2);
          }
          ngc += __popcll(cand2 & ~a1[q]);
        }
      }
    }
    if (!store2) continue;  // warp-uniform
    unsigned long long slot = warp_slots(ngc, &cntp[s % 3]);
    if (ngc == 0) continue;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      unsigned long long b = ch1[k];
      while (b) {
        const unsigned int v = 64u * k + __ffsll((long long)b) - 1;
        b &= b - 1;
        const unsigned long long hv = H + rtab[v];
        unsigned long long nb2[W];
#pragma unroll
        for (int q = 0; q < W; ++q) nb2[q] = nb1[q] | adj[(unsigned long long)v * W + q];
#pragma unroll
        for (int q = 0; q < W; ++q) {
          unsigned long long g = adj[(unsigned long long)v * W + q] & ~nb1[q] & ~a1[q];
          while (g) {
            const unsigned int w = 64u * q + __ffsll((long long)g) - 1;
            g &= g - 1;
            if (slot < ds) {
#pragma unroll
              for (int r = 0; r < W; ++r) {
                dB[r * ds + slot] = nb2[r];
                if (next_ok) nx += __popcll(adj[(unsigned long long)w * W + r] & ~nb2[r] & ~a1[r]);
              }
              dH[slot] = hv + rtab[w];
              dM[slot] = v1 | (w << 16);
            } else {
              set_err(p.ctl, kDevBounds, 5);
            }
            ++slot;
          }
        }
      }
    }
  }
  block_sum3_u64(nx, ncyc1, hacc, s_red);
  __syncthreads();
  unsigned long long z0 = 0, z1 = 0;
  block_sum3_u64(ncyc2, z0, z1, s_red);
  if (tid == 0) {
    if (nx) atomicAdd(&nxtp[s % 3], nx);
    if (ncyc1) atomicAdd(&p.hist[t + 1], ncyc1);
    if (ncyc2) atomicAdd(&p.hist[t + 2], ncyc2);
    if (hacc) atomicAdd(p.hash, hacc);
  }
}

// Single-graph bitset expansion with flattened output.  The per-path part (load B, H, M;
// cand = Adj(vt) & ~B, close = cand & Adj(v1), child = cand & ~Adj(v1)) is as above, but
// each path's B | Adj(vt), H and v1 are staged in shared memory and its children are
// listed as (path, vertex) entries.  The entries are then worked off with one entry per
// lane: a warp's child list takes its slots with one atomic and lane i writes slot
// base + i, so each plane is stored contiguously.  This replaces the per-lane loops over
// a path's children, whose cost was set by the lane with the most children.  Closings
// (a few per path) add h(C) = mix(H + r(v) + (t+1) gamma) in place, lane by lane.
template <int W, int P, int NT>
struct FlatSmem {
  static constexpr unsigned int CL = 64 * P > 256 ? 256 : 64 * P;  // list entries per warp
  unsigned long long nb[NT / 32][P * 32 * W];  // B | Adj(vt) per staged path
  unsigned long long h[NT / 32][P * 32];       // H per staged path
  unsigned int v1[NT / 32][P * 32];            // v1 per staged path
  unsigned int list[NT / 32][CL];              // entries: path << 8 | v
};

template <int W, int P, int NT>
__device__ __forceinline__ FlatSmem<W, P, NT>& flat_smem() {
  __shared__ FlatSmem<W, P, NT> fs;
  return fs;
}

template <Kind K, int NT>
__device__ __forceinline__ void process_bitset_flat(const EngineParams& p, const StepPlan& pl,
                                                    const unsigned long long* adj, const unsigned long long* rtab,
                                                    unsigned long long* s_red) {
  constexpr int W = KindTraits<K>::W;
  constexpr int P = KindTraits<K>::PF;
  constexpr unsigned int CL = FlatSmem<W, P, NT>::CL;
  FlatSmem<W, P, NT>& fs = flat_smem<W, P, NT>();
  const unsigned int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned long long* snb = fs.nb[wid];
  unsigned long long* sh = fs.h[wid];
  unsigned int* sv1 = fs.v1[wid];
  unsigned int* sl = fs.list[wid];
  const unsigned long long ss = pl.src_stride, ds = pl.dst_stride;
  const unsigned long long* sB = reinterpret_cast<const unsigned long long*>(p.arena + pl.src_base);
  const unsigned long long* sH = sB + W * ss;
  const unsigned int* sM = reinterpret_cast<const unsigned int*>(sH + ss);
  unsigned long long* dB = reinterpret_cast<unsigned long long*>(p.arena + pl.dst_base);
  unsigned long long* dH = dB + W * ds;
  unsigned int* dM = reinterpret_cast<unsigned int*>(dH + ds);
  const bool store = ds != 0;
  const unsigned int t = pl.t, L = p.L;
  const unsigned long long s = pl.s;
  const bool close_ok = t + 1 <= L, next_ok = t + 2 < L;
  const unsigned long long gam = (unsigned long long)(t + 1) * kGamma;
  unsigned long long hacc = 0;
  unsigned int nx = 0, ncyc = 0;  // per lane and step: 32 bits
  // (record indices relative to the step's first record and the child region: 32 bits, as
  // the planner keeps bitset frames under 2^32 records)
  const unsigned int ds32 = (unsigned int)min(ds, 0xFFFFFFFFull);
  const unsigned int nrec = (unsigned int)(pl.end - pl.begin);
  const unsigned long long* sB0 = sB + pl.begin;
  const unsigned long long* sH0 = sH + pl.begin;
  const unsigned int* sM0 = sM + pl.begin;
  const unsigned int T = gridDim.x * blockDim.x;
  const unsigned int gwarp = (wid * gridDim.x + blockIdx.x) * 32u;

  // list the set bits of m[j][k] (j < P, k < W), the children of the staged paths, as
  // entries, CL at a time, and write each chunk out with one entry per lane.  The warp's
  // slots come from one atomic, issued before the listing so that its round trip overlaps
  // it; lane i writes slot base + c0 + i, so each plane is stored contiguously.
  unsigned long long m[P][W];
  auto list_children = [&]() {
    unsigned int cnt = 0;
#pragma unroll
    for (int j = 0; j < P; ++j)
#pragma unroll
      for (int k = 0; k < W; ++k) cnt += __popcll(m[j][k]);
    unsigned int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    const unsigned int excl = incl - cnt, total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&p.ctl->cnt[s % 3], (unsigned long long)total);
    const unsigned int base32 = (unsigned int)__shfl_sync(0xffffffffu, base, 0);
    for (unsigned int c0 = 0; c0 < total; c0 += CL) {
      if (cnt && excl < c0 + CL && excl + cnt > c0) {
        unsigned int idx = excl;
#pragma unroll
        for (int j = 0; j < P; ++j)
#pragma unroll
          for (int k = 0; k < W; ++k) {
            unsigned long long b = m[j][k];
            while (b) {
              const unsigned int v = 64u * k + __ffsll((long long)b) - 1;
              b &= b - 1;
              if (idx >= c0 && idx < c0 + CL) sl[idx - c0] = (unsigned int)(j * 32 + lane) << 8 | v;
              ++idx;
            }
          }
      }
      __syncwarp();
      const unsigned int b0 = base32 + c0;
      const unsigned int n = min(CL, total - c0);
      for (unsigned int i = lane; i < n; i += 32) {
        const unsigned int e = sl[i], pj = e >> 8, v = e & 0xFFu;
        const unsigned int slot = b0 + i;
        if (slot < ds32) {
          const unsigned int v1 = sv1[pj];
#pragma unroll
          for (int q = 0; q < W; ++q) {
            const unsigned long long nb = snb[pj * W + q];
            dB[q * ds + slot] = nb;
            if (next_ok) nx += __popcll(adj[(unsigned long long)v * W + q] & ~nb & ~adj[(unsigned long long)v1 * W + q]);
          }
          dH[slot] = sh[pj] + rtab[v];
          dM[slot] = v1 | (v << 16);
        } else {
          set_err(p.ctl, kDevBounds, 1);
        }
      }
      __syncwarp();
    }
  };

  const unsigned int pf = p.pf >= 1 && p.pf <= (unsigned)P ? p.pf : (unsigned)P;
  for (unsigned int wb = gwarp; wb < nrec; wb += pf * T) {
    const unsigned int t0 = wb + lane;
    unsigned long long cm[P][W];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const unsigned int i = t0 + j * T;
      const bool valid = (unsigned)j < pf && i < nrec;
      unsigned long long B[W];
#pragma unroll
      for (int k = 0; k < W; ++k) B[k] = valid ? ldcg64(sB0 + k * ss + i) : ~0ull;
      const unsigned long long H = valid ? ldcg64(sH0 + i) : 0ull;
      const unsigned int M = valid ? ldcg32(sM0 + i) : 0u;
      const unsigned int v1 = M & 0xFFFFu, vt = M >> 16;
      const unsigned int pj = j * 32 + lane;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        const unsigned long long at = adj[(unsigned long long)vt * W + k];
        const unsigned long long a1 = adj[(unsigned long long)v1 * W + k];
        const unsigned long long cand = at & ~B[k];
        m[j][k] = store ? (cand & ~a1) : 0ull;
        cm[j][k] = close_ok ? (cand & a1) : 0ull;
        snb[pj * W + k] = B[k] | at;
      }
      sh[pj] = H;
      sv1[pj] = v1;
    }
    // closings <p, v> (a few per path): hashed in place, lane by lane
#pragma unroll
    for (int j = 0; j < P; ++j)
#pragma unroll
      for (int k = 0; k < W; ++k) {
        unsigned long long cb = cm[j][k];
        if (cb) {
          const unsigned long long H = sh[j * 32 + lane];
          do {
            const unsigned int v = 64u * k + __ffsll((long long)cb) - 1;
            cb &= cb - 1;
            ++ncyc;
            hacc += mix64(H + rtab[v] + gam);
          } while (cb);
        }
      }
    if (store) list_children();
  }
  unsigned long long nx64 = nx, ncyc64 = ncyc;
  block_sum3_u64(nx64, ncyc64, hacc, s_red);
  if (tid == 0) {
    if (nx64) atomicAdd(&p.ctl->nxt[s % 3], nx64);
    if (ncyc64) atomicAdd(&p.hist[t + 1], ncyc64);
    if (hacc) atomicAdd(p.hash, hacc);
  }
}

// Two levels in one step (single graph, bitset).  Level t is expanded as in the flattened
// form, but every candidate (closing or child) is listed once; the list is worked off
// P2*32 entries at a time: a candidate adjacent to v1 closes a cycle of t+1 vertices, any
// other is a child of level t+1, which is not stored.  Its own closings (cycles of t+2
// vertices) are hashed in place, and it is staged in shared memory with its blocked set
// B | Adj(vt) | Adj(v), H + r(v) and its child mask.  The staged children's children
// (level t+2) are then listed and stored in the flattened way, with their exact child
// counts summed for the next frame.
template <int W, int P, int NT>
struct FusedSmem {
  unsigned long long nb[NT / 32][P * 32 * W];  // staged children: blocked set of their children
  unsigned long long h[NT / 32][P * 32];       // their H'
  unsigned long long ch[NT / 32][P * 32 * W];  // child mask (stored paths of t+2 vertices)
  unsigned int v1[NT / 32][P * 32];
  unsigned int list[NT / 32][64 * P];  // level t+2 entries: slot << 8 | w
};

template <Kind K, int NT>
__device__ __forceinline__ void process_bitset_fused(const EngineParams& p, const StepPlan& pl,
                                                     const unsigned long long* adj, const unsigned long long* rtab,
                                                     unsigned long long* s_red) {
  constexpr int W = KindTraits<K>::W;
  constexpr int P = KindTraits<K>::PF, P2 = KindTraits<K>::PF2;
  constexpr unsigned int CL = FlatSmem<W, P, NT>::CL, CL2 = 64 * P2;
  FlatSmem<W, P, NT>& fs = flat_smem<W, P, NT>();
  __shared__ FusedSmem<W, P2, NT> fs2;
  const unsigned int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned long long* snb = fs.nb[wid];
  unsigned long long* sh = fs.h[wid];
  unsigned int* sv1 = fs.v1[wid];
  unsigned int* sl = fs.list[wid];
  unsigned long long* snb2 = fs2.nb[wid];
  unsigned long long* sh2 = fs2.h[wid];
  unsigned long long* sch2 = fs2.ch[wid];
  unsigned int* sv12 = fs2.v1[wid];
  unsigned int* sl2 = fs2.list[wid];
  const unsigned long long ss = pl.src_stride, ds = pl.dst_stride;
  const unsigned long long* sB = reinterpret_cast<const unsigned long long*>(p.arena + pl.src_base);
  const unsigned long long* sH = sB + W * ss;
  const unsigned int* sM = reinterpret_cast<const unsigned int*>(sH + ss);
  unsigned long long* dB = reinterpret_cast<unsigned long long*>(p.arena + pl.dst_base);
  unsigned long long* dH = dB + W * ds;
  unsigned int* dM = reinterpret_cast<unsigned int*>(dH + ds);
  const unsigned int t = pl.t, L = p.L;
  const unsigned long long s = pl.s;
  // level t+1 is stored in the single-level form (t+1 < L' holds for a fused step)
  const bool close2_ok = t + 2 <= L, store2 = ds != 0, next_ok = t + 3 < L;
  const unsigned long long gam1 = (unsigned long long)(t + 1) * kGamma, gam2 = (unsigned long long)(t + 2) * kGamma;
  unsigned long long hacc = 0;
  unsigned int nx = 0, ncyc1 = 0, ncyc2 = 0;  // per lane and step: 32 bits
  // (record indices relative to the step's first record and the child region: 32 bits, as
  // the planner keeps bitset frames under 2^32 records)
  const unsigned int ds32 = (unsigned int)min(ds, 0xFFFFFFFFull);
  const unsigned int nrec = (unsigned int)(pl.end - pl.begin);
  const unsigned long long* sB0 = sB + pl.begin;
  const unsigned long long* sH0 = sH + pl.begin;
  const unsigned int* sM0 = sM + pl.begin;
  const unsigned int T = gridDim.x * blockDim.x;
  const unsigned int gwarp = (wid * gridDim.x + blockIdx.x) * 32u;

  auto scan = [&](unsigned int cnt, unsigned int& excl, unsigned int& total) {
    unsigned int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    excl = incl - cnt;
    total = __shfl_sync(0xffffffffu, incl, 31);
  };

  // ---- level t+2: list the staged children's child masks and write the entries out,
  // CL2 at a time (slots from one atomic per list, issued before the listing)
  auto list2_children = [&]() {
    unsigned int cnt = 0;
#pragma unroll
    for (int j = 0; j < P2; ++j)
#pragma unroll
      for (int k = 0; k < W; ++k) cnt += __popcll(sch2[(j * 32 + lane) * W + k]);
    unsigned int excl, total;
    scan(cnt, excl, total);
    if (total == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&p.ctl->cnt[s % 3], (unsigned long long)total);
    const unsigned int base32 = (unsigned int)__shfl_sync(0xffffffffu, base, 0);
    for (unsigned int c0 = 0; c0 < total; c0 += CL2) {
      if (cnt && excl < c0 + CL2 && excl + cnt > c0) {
        unsigned int idx = excl;
#pragma unroll
        for (int j = 0; j < P2; ++j)
#pragma unroll
          for (int k = 0; k < W; ++k) {
            unsigned long long b = sch2[(j * 32 + lane) * W + k];
            while (b) {
              const unsigned int w = 64u * k + __ffsll((long long)b) - 1;
              b &= b - 1;
              if (idx >= c0 && idx < c0 + CL2) sl2[idx - c0] = (unsigned int)(j * 32 + lane) << 8 | w;
              ++idx;
            }
          }
      }
      __syncwarp();
      const unsigned int b0 = base32 + c0;
      const unsigned int n = min(CL2, total - c0);
      for (unsigned int i = lane; i < n; i += 32) {
        const unsigned int e = sl2[i], c = e >> 8, w = e & 0xFFu;
        const unsigned int slot = b0 + i;
        if (slot < ds32) {
          const unsigned int v1 = sv12[c];
#pragma unroll
          for (int q = 0; q < W; ++q) {
            const unsigned long long nb = snb2[c * W + q];
            dB[q * ds + slot] = nb;
            if (next_ok)
              nx += __popcll(adj[(unsigned long long)w * W + q] & ~nb & ~adj[(unsigned long long)v1 * W + q]);
          }
          dH[slot] = sh2[c] + rtab[w];
          dM[slot] = v1 | (w << 16);
        } else {
          set_err(p.ctl, kDevBounds, 4);
        }
      }
      __syncwarp();
    }
  };

  // ---- level t+1: the candidates listed in sl[0, n), P2*32 at a time
  auto expand_children = [&](unsigned int n) {
    __syncwarp();
    for (unsigned int r0 = 0; r0 < n; r0 += P2 * 32) {
#pragma unroll
      for (int j = 0; j < P2; ++j) {
        const unsigned int slot = j * 32 + lane, i = r0 + slot;
        unsigned long long mg[W];
#pragma unroll
        for (int k = 0; k < W; ++k) mg[k] = 0ull;
        if (i < n) {
          const unsigned int e = sl[i], pj = e >> 8, v = e & 0xFFu;
          const unsigned int v1 = sv1[pj];
          const unsigned long long hv = sh[pj] + rtab[v];
          if ((adj[(unsigned long long)v1 * W + (v >> 6)] >> (v & 63u)) & 1ull) {
            ++ncyc1;
            hacc += mix64(hv + gam1);
          } else {
#pragma unroll
            for (int k = 0; k < W; ++k) {
              const unsigned long long nb1 = snb[pj * W + k];  // the child's blocked set
              const unsigned long long av = adj[(unsigned long long)v * W + k];
              const unsigned long long a1 = adj[(unsigned long long)v1 * W + k];
              const unsigned long long cand = av & ~nb1;
              mg[k] = store2 ? (cand & ~a1) : 0ull;
              snb2[slot * W + k] = nb1 | av;
              // closings of t+2 vertices: hashed in place
              unsigned long long cb = close2_ok ? (cand & a1) : 0ull;
              while (cb) {
                const unsigned int w = 64u * k + __ffsll((long long)cb) - 1;
                cb &= cb - 1;
                ++ncyc2;
                hacc += mix64(hv + rtab[w] + gam2);
              }
            }
            sh2[slot] = hv;
            sv12[slot] = v1;
          }
        }
#pragma unroll
        for (int k = 0; k < W; ++k) sch2[slot * W + k] = mg[k];
      }
      __syncwarp();
      if (store2) list2_children();
    }
  };

  // ---- level t: load, stage, list every candidate (closing or child)
  unsigned long long m[P][W];
  auto list_and_work = [&]() {
    unsigned int cnt = 0;
#pragma unroll
    for (int j = 0; j < P; ++j)
#pragma unroll
      for (int k = 0; k < W; ++k) cnt += __popcll(m[j][k]);
    unsigned int excl, total;
    scan(cnt, excl, total);
    for (unsigned int c0 = 0; c0 < total; c0 += CL) {
      if (cnt && excl < c0 + CL && excl + cnt > c0) {
        unsigned int idx = excl;
#pragma unroll
        for (int j = 0; j < P; ++j)
#pragma unroll
          for (int k = 0; k < W; ++k) {
            unsigned long long b = m[j][k];
            while (b) {
              const unsigned int v = 64u * k + __ffsll((long long)b) - 1;
              b &= b - 1;
              if (idx >= c0 && idx < c0 + CL) sl[idx - c0] = (unsigned int)(j * 32 + lane) << 8 | v;
              ++idx;
            }
          }
      }
      expand_children(min(CL, total - c0));
    }
  };

  const unsigned int pf = p.pf >= 1 && p.pf <= (unsigned)P ? p.pf : (unsigned)P;
  for (unsigned int wb = gwarp; wb < nrec; wb += pf * T) {
    const unsigned int t0 = wb + lane;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const unsigned int i = t0 + j * T;
      const bool valid = (unsigned)j < pf && i < nrec;
      unsigned long long B[W];
#pragma unroll
      for (int k = 0; k < W; ++k) B[k] = valid ? ldcg64(sB0 + k * ss + i) : ~0ull;
      const unsigned long long H = valid ? ldcg64(sH0 + i) : 0ull;
      const unsigned int M = valid ? ldcg32(sM0 + i) : 0u;
      const unsigned int v1 = M & 0xFFFFu, vt = M >> 16;
      const unsigned int pj = j * 32 + lane;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        const unsigned long long at = adj[(unsigned long long)vt * W + k];
        m[j][k] = at & ~B[k];  // candidates: closings and children of t+1 vertices
        snb[pj * W + k] = B[k] | at;
      }
      sh[pj] = H;
      sv1[pj] = v1;
    }
    list_and_work();
  }
  // hist[t+1] and hist[t+2]: two block sums
  unsigned long long nx64 = nx, ncyc1_64 = ncyc1, ncyc2_64 = ncyc2;
  block_sum3_u64(nx64, ncyc1_64, hacc, s_red);
  __syncthreads();
  unsigned long long z0 = 0, z1 = 0;
  block_sum3_u64(ncyc2_64, z0, z1, s_red);
  if (tid == 0) {
    if (nx64) atomicAdd(&p.ctl->nxt[s % 3], nx64);
    if (ncyc1_64) atomicAdd(&p.hist[t + 1], ncyc1_64);
    if (ncyc2_64) atomicAdd(&p.hist[t + 2], ncyc2_64);
    if (hacc) atomicAdd(p.hash, hacc);
  }
}

// The batch form of the flattened expansion (records of many graphs in one frontier; M
// holds v1, vt, t and the graph's slot g, whose rows and r-table sit at g * 64).  Per-path
// statistics (paths expanded, children, closings and their hashes per (slot, length)) are
// accumulated in lane order as runs of one key, as in the per-lane form.  A path closes
// few cycles (about one for every five paths stored), so each lane hashes its own paths'
// closings in place.  The children are worked off one per lane: child i of a round belongs
// to the last lane whose first child index is at most i (a binary search over the lanes'
// exclusive prefix counts, by shuffles), and is the k-th set bit of that lane's masks.
//
// Work distribution: a warp takes contiguous chunks of the step's records from a step
// counter (one atomic per chunk), so its rounds mostly stay inside one graph's run of
// records while the chunks balance the load between warps.  Each record carries its exact
// child count (N, written with it), so the warp reserves the child slots of a whole chunk
// with one atomic before expanding it: a single counter taking one atomic per round was
// the hot spot of the whole grid.  The rows, r-table and L' of the graph a warp is working
// on are staged in the warp's shared memory when the graph changes; records of any other
// graph in the same round read them from global memory.
template <int NT>
__device__ __forceinline__ void process_multi_flat(const EngineParams& p, const StepPlan& pl,
                                                   const unsigned long long* adj, const unsigned long long* rtab) {
  constexpr int P = KindTraits<Kind::Multi>::P;
  static_assert(P == 2, "the batch form takes two paths per lane and round");
  __shared__ unsigned long long s_nb[NT / 32][P * 32];  // B | Adj(vt) per staged path
  __shared__ unsigned long long s_h[NT / 32][P * 32];   // H per staged path
  __shared__ unsigned int s_meta[NT / 32][P * 32];
  __shared__ unsigned long long s_gadj[NT / 32][64];
  __shared__ unsigned long long s_grt[NT / 32][64];
  __shared__ unsigned long long s_rb[NT / 32][2][P * 32];  // records of this round and the next
  __shared__ unsigned long long s_rh[NT / 32][2][P * 32];
  __shared__ unsigned int s_rm[NT / 32][2][P * 32];
  const unsigned int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned long long* snb = s_nb[wid];
  unsigned long long* sh = s_h[wid];
  unsigned int* smeta = s_meta[wid];  // v1 | t << 6 | g << 12 | (t + 2 < L'_g) << 31
  unsigned long long* ga = s_gadj[wid];
  unsigned long long* gr = s_grt[wid];
  const unsigned long long ss = pl.src_stride, ds = pl.dst_stride;
  const unsigned long long* sB = reinterpret_cast<const unsigned long long*>(p.arena + pl.src_base);
  const unsigned long long* sH = sB + ss;
  const unsigned int* sM = reinterpret_cast<const unsigned int*>(sH + ss);
  const unsigned char* sN = reinterpret_cast<const unsigned char*>(sM + ss);
  // (record indices below are relative to the step's first record and to the child region:
  // 32 bits, as the planner keeps batch frames under 2^32 records)
  unsigned long long* dB = reinterpret_cast<unsigned long long*>(p.arena + pl.dst_base);
  unsigned long long* dH = dB + ds;
  unsigned int* dM = reinterpret_cast<unsigned int*>(dH + ds);
  unsigned char* dN = reinterpret_cast<unsigned char*>(dM + ds);
  const bool store = ds != 0;
  const unsigned int ds32 = (unsigned int)min(ds, 0xFFFFFFFFull);
  const unsigned long long s = pl.s;
  unsigned int nx = 0;  // children of this lane's stored children (fits 32 bits per lane and step)
  StatRun run;
  run.key = 0xFFFFFFFFu;
  unsigned int cg = 0xFFFFFFFFu;  // graph staged in ga / gr
  unsigned int cL = 0;            // its L'
  auto A = [&](unsigned int g, unsigned int v) -> unsigned long long {
    return g == cg ? ga[v] : __ldg(adj + (unsigned long long)g * 64ull + v);
  };
  auto R = [&](unsigned int g, unsigned int v) -> unsigned long long {
    return g == cg ? gr[v] : __ldg(rtab + (unsigned long long)g * 64ull + v);
  };

  unsigned long long m[P];
  unsigned int cnext = 0, cend_slot = 0;  // the chunk's reserved child slots (warp-uniform)
  // The round's children <p, v> (masks m[0], m[1] of each lane's two paths) take the next
  // slots of the chunk's range, in lane order.
  auto children = [&]() {
    const unsigned int c0n = __popcll(m[0]);
    const unsigned int cnt = c0n + __popcll(m[1]);
    unsigned int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    const unsigned int excl = incl - cnt, n = __shfl_sync(0xffffffffu, incl, 31);
    const unsigned int base = cnext;
    cnext += n;
    __syncwarp();  // the staged paths (snb, sh, smeta) of every lane
    for (unsigned int w0 = 0; w0 < n; w0 += 32) {
      const unsigned int i = w0 + lane;
      // owner: the last lane whose first child index is at most i (a lane without children
      // shares its index with the next lane, so the last such lane has child i)
      unsigned int o = 0, eo = 0;
#pragma unroll
      for (unsigned int st = 16; st >= 1; st >>= 1) {
        const unsigned int e = __shfl_sync(0xffffffffu, excl, o + st);
        if (e <= i) {
          o += st;
          eo = e;
        }
      }
      const unsigned long long b0 = __shfl_sync(0xffffffffu, m[0], o), b1 = __shfl_sync(0xffffffffu, m[1], o);
      const unsigned int c0o = __shfl_sync(0xffffffffu, c0n, o);
      if (i < n) {
        unsigned int k = i - eo, j = 0;
        unsigned long long b = b0;
        if (k >= c0o) {
          k -= c0o;
          j = 1;
          b = b1;
        }
        for (; k; --k) b &= b - 1;  // the k-th set bit of the path's child mask
        const unsigned int v = __ffsll((long long)b) - 1, pj = j * 32u + o;
        const unsigned int meta = smeta[pj], v1 = meta & 63u, tt = (meta >> 6) & 63u, g = (meta >> 12) & 0x7FFFFu;
        const unsigned int slot = base + i;
        if (slot < ds32) {
          const unsigned long long nb = snb[pj];
          dB[slot] = nb;
          dH[slot] = sh[pj] + R(g, v);
          dM[slot] = v1 | (v << 6) | ((tt + 1) << 12) | (g << 18);
          const unsigned int nc = (meta >> 31) ? __popcll(A(g, v) & ~nb & ~A(g, v1)) : 0u;
          dN[slot] = (unsigned char)nc;
          nx += nc;
        } else {
          set_err(p.ctl, kDevBounds, 1);
        }
      }
    }
    __syncwarp();
  };

  const unsigned int pf = p.pf >= 1 && p.pf <= (unsigned)P ? p.pf : (unsigned)P;
  const unsigned int RW = pf * 32;  // records per warp round
  const unsigned int total = (unsigned int)(pl.end - pl.begin);  // (below 2^32, see plan_step)
  const unsigned int nwarps = gridDim.x * (NT / 32);
  // chunks of about a quarter of a warp's share, between 1 and 32 rounds
  unsigned int chunk = (total / (nwarps * 4) + RW - 1) / RW * RW;
  chunk = chunk < RW ? RW : (chunk > 32u * RW ? 32u * RW : chunk);
  // the step's records, indexed from its first one
  const unsigned long long* sB0 = sB + pl.begin;
  const unsigned long long* sH0 = sH + pl.begin;
  const unsigned int* sM0 = sM + pl.begin;
  const unsigned char* sN0 = sN + pl.begin;
  for (;;) {
    unsigned long long c64 = 0;
    if (lane == 0) c64 = atomicAdd(&p.ctl->take[s % 3], (unsigned long long)chunk);
    c64 = __shfl_sync(0xffffffffu, c64, 0);
    if (c64 >= total) break;
    const unsigned int c0 = (unsigned int)c64;
    const unsigned int cend = min(c0 + chunk, total);
    // the chunk's children (the records' exact child counts) take one range of slots
    if (store) {
      unsigned int nch = 0;
      for (unsigned int i = c0 + lane; i < cend; i += 32) nch += ldcg8(sN0 + i);
      nch = __reduce_add_sync(0xffffffffu, nch);
      unsigned long long b = 0;
      if (lane == 0 && nch) b = atomicAdd(&p.ctl->cnt[s % 3], (unsigned long long)nch);
      cnext = (unsigned int)__shfl_sync(0xffffffffu, b, 0);
      cend_slot = cnext + nch;
    }
    // the records of a round are copied into this warp's shared memory by cp.async while
    // the round before is expanded (each lane copies, then reads, its own records)
    auto prefetch = [&](unsigned int w0, unsigned int buf) {
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const unsigned int i = w0 + lane + j * 32u;
        if ((unsigned)j < pf && i < cend) {
          cp_async8(&s_rb[wid][buf][j * 32 + lane], sB0 + i);
          cp_async8(&s_rh[wid][buf][j * 32 + lane], sH0 + i);
          cp_async4(&s_rm[wid][buf][j * 32 + lane], sM0 + i);
        }
      }
      cp_async_commit();
    };
    unsigned int buf = 0;
    prefetch(c0, 0);
    for (unsigned int wb = c0; wb < cend; wb += RW, buf ^= 1u) {
      if (wb + RW < cend) prefetch(wb + RW, buf ^ 1u);
      else cp_async_commit();  // (an empty group: the wait below still means "this round")
      cp_async_wait_1();
      // the graph of the round's first record (always valid): stage it if it changed
      const unsigned int g0 = __shfl_sync(0xffffffffu, s_rm[wid][buf][lane], 0) >> 18;
      if (g0 != cg) {
        __syncwarp();
        ga[lane] = __ldg(adj + (unsigned long long)g0 * 64ull + lane);
        ga[lane + 32] = __ldg(adj + (unsigned long long)g0 * 64ull + lane + 32);
        gr[lane] = __ldg(rtab + (unsigned long long)g0 * 64ull + lane);
        gr[lane + 32] = __ldg(rtab + (unsigned long long)g0 * 64ull + lane + 32);
        cL = p.Lg[g0];
        cg = g0;
        __syncwarp();
      }
      const unsigned int t0 = wb + lane;
      unsigned long long ch[P];
      unsigned int key[P], nc[P], nk[P];
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const unsigned int i = t0 + j * 32u;
        const bool valid = (unsigned)j < pf && i < cend;
        const unsigned long long B = valid ? s_rb[wid][buf][j * 32 + lane] : ~0ull;
        const unsigned long long H = valid ? s_rh[wid][buf][j * 32 + lane] : 0ull;
        const unsigned int M = valid ? s_rm[wid][buf][j * 32 + lane] : 0u;
        const unsigned int v1 = M & 63u, vt = (M >> 6) & 63u, tt = (M >> 12) & 63u, g = M >> 18;
        const unsigned int Lr = valid ? (g == cg ? cL : p.Lg[g]) : 0u;
        const unsigned long long at = A(g, vt), a1 = A(g, v1);
        const unsigned long long cand = at & ~B;
        m[j] = (tt + 1 <= Lr) ? (cand & a1) : 0ull;
        ch[j] = (store && tt + 1 < Lr) ? (cand & ~a1) : 0ull;
        const unsigned int pj = j * 32 + lane;
        snb[pj] = B | at;
        sh[pj] = H;
        smeta[pj] = v1 | (tt << 6) | (g << 12) | ((tt + 2 < Lr) ? 0x80000000u : 0u);
        key[j] = valid ? (g << 6 | tt) : 0xFFFFFFFFu;
        nc[j] = __popcll(m[j]);
        nk[j] = __popcll(ch[j]);
      }
      // the closings <p, v>, hashed in place: h(C) = mix(H + r(v) + (t+1) gamma), one bit
      // of either path's mask per iteration
      static_assert(P == 2, "the closing loop takes two paths per lane");
      unsigned long long hs0 = 0, hs1 = 0;
      {
        unsigned long long b0 = m[0], b1 = m[1];
        if (b0 | b1) {
          const unsigned long long hb0 = sh[lane] + (unsigned long long)((key[0] & 63u) + 1u) * kGamma;
          const unsigned long long hb1 = sh[32 + lane] + (unsigned long long)((key[1] & 63u) + 1u) * kGamma;
          do {
            const bool f = b0 != 0;
            const unsigned long long b = f ? b0 : b1;
            const unsigned int v = __ffsll((long long)b) - 1;
            const unsigned long long h = mix64((f ? hb0 : hb1) + R((f ? key[0] : key[1]) >> 6, v));
            if (f) {
              hs0 += h;
              b0 &= b0 - 1;
            } else {
              hs1 += h;
              b1 &= b1 - 1;
            }
          } while (b0 | b1);
        }
      }
      // per (slot, length) counts and closing hashes, as runs of one key
#pragma unroll
      for (int j = 0; j < P; ++j) {
        const unsigned int k = key[j];
        const unsigned long long hj = j == 0 ? hs0 : hs1;
        const bool v = k != 0xFFFFFFFFu;
        const bool m0 = v && k == run.key;
        if (m0) run.add(nc[j], nk[j], hj);
        const unsigned int rest = __ballot_sync(0xffffffffu, v && !m0);
        if (rest) {
          run.flush(p, s);
          run.key = __shfl_sync(0xffffffffu, k, 31 - __clz(rest));
          const bool m1 = v && !m0 && k == run.key;
          if (m1) run.add(nc[j], nk[j], hj);
          unsigned int pending = __ballot_sync(0xffffffffu, v && !m0 && !m1);
          while (pending) {
            const int leader = __ffs(pending) - 1;
            const unsigned int lk = __shfl_sync(0xffffffffu, k, leader);
            const bool mine = k == lk;
            const unsigned int grp = __ballot_sync(0xffffffffu, mine);
            StatRun one;
            one.key = lk;
            if (mine) one.add(nc[j], nk[j], hj);
            one.flush(p, s);
            pending &= ~grp;
          }
        }
      }
      if (store) {
#pragma unroll
        for (int j = 0; j < P; ++j) m[j] = ch[j];
        children();
      }
    }
    // (the children listed equal the child counts the records carry; a mismatch would be a
    // bug, reported instead of writing into another chunk's slots)
    if (store && cnext != cend_slot && lane == 0) set_err(p.ctl, kDevBounds, 6);
  }
  run.flush(p, s);
  const unsigned long long tot = warp_sum_u64((unsigned long long)nx);
  if (lane == 0 && tot) atomicAdd(&p.ctl->nxt[s % 3], tot);
}

// ------------------------------------------------------------------ CSR expansion

// CSR records: the path's relabelled ids in order, as u16, padded with 0xFFFF (never a
// vertex id) to csr_rec_u16(t) = a multiple of 8 entries, so a record is read and written
// with 16-byte vector accesses.
__device__ __forceinline__ unsigned int rec_id(const unsigned int* row, unsigned int k) {
  const unsigned int x = row[k >> 1];
  return (k & 1) ? (x >> 16) : (x & 0xFFFFu);
}

// Algorithm 3 on CSR with the path as a vertex list.  Candidate v of Adj(vt):
//   label test   v > v2 (relabelled ids are label ranks), v != v_{t-1} (the only vertex
//                of a stored chordless path adjacent to vt);
//   chord test   no w in Adj(v) lies on v2..v_{t-1};
//   close test   v1 in Adj(v) gives a cycle of t+1 vertices, otherwise a child path.
// Both tests start from 128-bit signatures (sig_bit): when nsig(v) shares no bit with the
// path's interior signature and lacks v1's bit, v is a child with no scan of Adj(v);
// otherwise Adj(v) is scanned, and a neighbour whose bit is in the interior signature is
// compared with the stored ids.  When this step stores no children (t + 1 = L'), only
// closings count, and a path whose end vertices v1 and vt have disjoint neighbour
// signatures (no common neighbour) has no candidate at all.
//
// Warp-cooperative: a warp stages its 32 paths (rows of packed id pairs, odd stride) in
// shared memory, then works through the flattened list of (path, candidate) pairs, one
// pair per lane per round; the pair's path comes from the warp's prefix sums of candidate
// counts.  Pairs the signatures settle are done in that round; the others go to a
// per-warp queue that is worked off with every lane on one queued pair, so the scans of
// Adj(v) do not leave most lanes idle.  The records of the warp's next 32 paths are loaded
// into registers while the current ones are processed, and the ones after that are
// prefetched into L2 by the bulk-copy engine.  Accepted children go to a per-warp list
// (owner lane, vertex); the list takes its slots with one atomic and is written out with
// lane j writing child j, so a warp stores consecutive whole records.  CAP bounds the
// staged path length (16 or 32 vertices).
__device__ __forceinline__ bool sig_test(unsigned long long s0, unsigned long long s1, unsigned int b) {
  return (((b & 64u) ? s1 : s0) >> (b & 63u)) & 1ull;
}
// Is w one of the ids packed in row[0..nw)?  (v1 and vt are excluded by the caller; the
// 0xFFFF padding never equals a vertex id.)
__device__ __forceinline__ bool on_path(const unsigned int* row, unsigned int nw, unsigned int w) {
  const unsigned int ww = w | (w << 16);
  unsigned int any = 0;
  for (unsigned int q = 0; q < nw; ++q) {
    const unsigned int x = row[q] ^ ww;  // a zero 16-bit lane marks an equal id
    any |= (x - 0x00010001u) & ~x & 0x80008000u;
  }
  return any != 0;
}

// Per-warp shared memory of the CSR loops: staged rows, child list, queued exact tests.
// One buffer per block, sized for the kind's largest CAP, serves every CAP (a step runs
// one form, and steps are separated by barriers).
template <int CAP>
struct CsrSmem {
  static constexpr int RS = CAP / 2 + 1;
  unsigned int path[kMaxThreads / 32][32 * RS];
  unsigned int child[kMaxThreads / 32][128];
  unsigned int exact[kMaxThreads / 32][64];
};
template <int MAXCAP>
__device__ __forceinline__ unsigned char* csr_smem_raw() {
  __shared__ __align__(16) unsigned char raw[sizeof(CsrSmem<MAXCAP>)];
  return raw;
}
template <int CAP, int MAXCAP>
__device__ __forceinline__ CsrSmem<CAP>& csr_smem() {
  static_assert(CAP <= MAXCAP, "a CSR form's staging must fit the kind's buffer");
  return *reinterpret_cast<CsrSmem<CAP>*>(csr_smem_raw<MAXCAP>());
}

template <int CAP, int MAXCAP>
__device__ __forceinline__ void process_csr_coop(const EngineParams& p, const StepPlan& pl,
                                                 const unsigned int* nrow, const unsigned short* ncol,
                                                 const unsigned long long* nsig, const unsigned long long* rtab) {
  constexpr int NP = CAP / 2, RS = NP + 1;  // packed words per row, row stride (odd)
  constexpr int NQ = CAP / 8;               // uint4 per staged row
  constexpr unsigned int CL = 128;          // child list entries per warp
  constexpr unsigned int CX = 64;           // queued exact tests per warp
  CsrSmem<CAP>& sm = csr_smem<CAP, MAXCAP>();
  const unsigned int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned int lt_mask = (1u << lane) - 1u;
  unsigned int* sp = sm.path[wid];
  unsigned int* sc = sm.child[wid];
  unsigned int* sx = sm.exact[wid];
  const unsigned int t = pl.t, L = p.L;
  const unsigned int nv = csr_rec_u16(t) / 8, nv2 = csr_rec_u16(t + 1) / 8;  // uint4 per record
  const unsigned int nw = (t + 1) / 2;                                         // words holding ids
  const uint4* S = reinterpret_cast<const uint4*>(p.arena + pl.src_base);
  uint4* D = reinterpret_cast<uint4*>(p.arena + pl.dst_base);
  const ulonglong2* NS = reinterpret_cast<const ulonglong2*>(nsig);
  const unsigned long long ds = pl.dst_stride;
  const bool store = ds != 0;
  const bool close_ok = t + 1 <= L, bound_ok = t + 2 < L;
  const unsigned long long s = pl.s;
  unsigned long long ncyc = 0, hacc = 0, nbound = 0;
  const unsigned long long wstep = (unsigned long long)gridDim.x * (blockDim.x >> 5) * 32;
  unsigned long long w0 = pl.begin + ((unsigned long long)wid * gridDim.x + blockIdx.x) * 32;
  uint4 nx[NQ];
  auto fetch = [&](unsigned long long base) {
    const unsigned long long i = base + lane;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      nx[q] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
      if (i < pl.end && (unsigned)q < nv) nx[q] = __ldcg(S + i * nv + q);
    }
  };
  auto prefetch = [&](unsigned long long base) {
    if (lane == 0 && base < pl.end) {
      const unsigned long long k = min(32ull, pl.end - base);
      bulk_prefetch_l2(S + base * nv, (unsigned int)(k * nv * 16));
    }
  };
  // the child list: slots from one atomic, record j written by lane j % 32
  unsigned int nchild = 0;
  auto flush = [&]() {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&p.ctl->cnt[s % 3], (unsigned long long)nchild);
    base = __shfl_sync(0xffffffffu, base, 0);
    const unsigned int tw = t >> 1, sh = (t & 1) * 16;
    for (unsigned int j = lane; j < nchild; j += 32) {
      const unsigned int e = sc[j], v = e & 0xFFFFu;
      const unsigned int* orow = sp + (e >> 16) * RS;
      const unsigned long long slot = base + j;
      if (slot < ds) {
        for (unsigned int q = 0; q < nv2; ++q) {
          unsigned int w4[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const unsigned int wi = 4 * q + c;
            unsigned int x = wi < (unsigned)NP ? orow[wi] : 0xFFFFFFFFu;
            if (wi == tw) x = (x & ~(0xFFFFu << sh)) | (v << sh);
            w4[c] = x;
          }
          D[slot * nv2 + q] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
        if (bound_ok) nbound += nrow[v + 1] - nrow[v] - 1;  // its candidates: Adj(v) minus v_t
      } else {
        set_err(p.ctl, kDevBounds, 3);
      }
    }
    if (p.cyc_stream && t + 2 <= L) {  // streamed lists: the children's closing bound
      unsigned int k = 0;
      for (unsigned int j = lane; j < nchild; j += 32) {
        const unsigned int e = sc[j];
        const unsigned int* orow = sp + (e >> 16) * RS;
        k += closing_bound(nrow, ncol, nsig, e & 0xFFFFu, orow[0] & 0xFFFFu, rec_id(orow, t - 1));
      }
      k = __reduce_add_sync(0xffffffffu, k);
      if (lane == 0 && k) atomicAdd(&p.ctl->ncl[s % 3], (unsigned long long)k);
    }
    nchild = 0;
    __syncwarp();
  };
  auto add_children = [&](bool is_child, unsigned int own, unsigned int v) {
    const unsigned int bal = __ballot_sync(0xffffffffu, is_child);
    if (nchild + __popc(bal) > CL) flush();
    if (is_child) sc[nchild + __popc(bal & lt_mask)] = own << 16 | v;
    nchild += __popc(bal);
    __syncwarp();
  };

  if (w0 < pl.end) fetch(w0);
  prefetch(w0 + wstep);
  for (; w0 < pl.end; w0 += wstep) {
    const bool valid = w0 + lane < pl.end;
    unsigned int* row = sp + lane * RS;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      row[4 * q] = nx[q].x;
      row[4 * q + 1] = nx[q].y;
      row[4 * q + 2] = nx[q].z;
      row[4 * q + 3] = nx[q].w;
    }
    if (w0 + wstep < pl.end) fetch(w0 + wstep);
    prefetch(w0 + 2 * wstep);
    unsigned int v12 = 0xFFFF0000u, vtp = 0, rb = 0, cnt = 0;  // v1 | v2 << 16, vt | v_{t-1} << 16
    unsigned long long sg0 = 0, sg1 = 0;                      // interior signature
    if (valid) {
      v12 = row[0];
      const unsigned int vt = rec_id(row, t - 1);
      vtp = vt | rec_id(row, t - 2) << 16;
      rb = nrow[vt];
      cnt = nrow[vt + 1] - rb;
      if (!store && cnt) {
        // only closings count: some neighbour of vt must also neighbour v1
        const ulonglong2 a = NS[vt], c = NS[v12 & 0xFFFFu];
        if (((a.x & c.x) | (a.y & c.y)) == 0) cnt = 0;
      }
      if (cnt && store)
        for (unsigned int k = 1; k + 1 < t; ++k) {
          const unsigned int b = sig_bit(rec_id(row, k));
          if (b & 64u) sg1 |= 1ull << (b & 63u); else sg0 |= 1ull << (b & 63u);
        }
    }
    __syncwarp();
    unsigned int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    const unsigned int excl = incl - cnt, total = __shfl_sync(0xffffffffu, incl, 31);

    // queued exact tests: lane j takes entry j (owner lane << 16 | v)
    unsigned int nexact = 0;
    auto run_exact = [&]() {
      for (unsigned int r0 = 0; r0 < nexact; r0 += 32) {
        const bool act = r0 + lane < nexact;
        const unsigned int e = act ? sx[r0 + lane] : 0u;
        const unsigned int own = e >> 16, v = e & 0xFFFFu;
        const unsigned int o_v12 = __shfl_sync(0xffffffffu, v12, own);
        const unsigned int o_vtp = __shfl_sync(0xffffffffu, vtp, own);
        const unsigned long long o_sg0 = __shfl_sync(0xffffffffu, sg0, own);
        const unsigned long long o_sg1 = __shfl_sync(0xffffffffu, sg1, own);
        const unsigned int o_v1 = o_v12 & 0xFFFFu, o_v2 = o_v12 >> 16, o_vt = o_vtp & 0xFFFFu;
        const unsigned int* orow = sp + own * RS;
        bool is_child = false;
        if (act) {
          bool close = false, chord = false;
          const unsigned int f0 = nrow[v], e1 = nrow[v + 1];
          if (store) {
            for (unsigned int f = f0; f < e1; ++f) {
              const unsigned int w = ncol[f];
              if (w < o_v2 || w == o_vt) continue;
              if (w == o_v1) {
                close = true;
                continue;
              }
              if (sig_test(o_sg0, o_sg1, sig_bit(w)) && on_path(orow, nw, w)) {
                chord = true;
                break;
              }
            }
          } else {
            // only a closing counts: v1 in Adj(v) first (sorted row, stop at the first
            // id >= v1), then the chord test against the staged ids
            unsigned int f = f0;
            while (f < e1 && ncol[f] < o_v1) ++f;
            close = f < e1 && ncol[f] == o_v1;
            for (f = f0; close && !chord && f < e1; ++f) {
              const unsigned int w = ncol[f];
              if (w < o_v2 || w == o_vt || w == o_v1) continue;
              chord = on_path(orow, nw, w);
            }
          }
          if (!chord) {
            if (close) {
              if (close_ok) {
                ++ncyc;
                unsigned long long hs = rtab[v];
                for (unsigned int j = 0; j < t; ++j) hs += rtab[rec_id(orow, j)];
                hacc += mix64(hs + (unsigned long long)(t + 1) * kGamma);
                if (p.cyc_vert)
                  emit_cycle(p, t + 1, [&](unsigned int j) -> unsigned int { return j < t ? rec_id(orow, j) : v; });
              }
            } else {
              is_child = store;
            }
          }
        }
        if (store) add_children(is_child, own, v);
      }
      nexact = 0;
      __syncwarp();
    };

    for (unsigned int r0 = 0; r0 < total; r0 += 32) {
      const unsigned int k = r0 + lane;
      // owner: the last lane whose exclusive offset is <= k
      unsigned int own = 0;
#pragma unroll
      for (int b = 16; b >= 1; b >>= 1) {
        const unsigned int e = __shfl_sync(0xffffffffu, excl, (own + b) & 31);
        if (own + b < 32 && e <= k) own += b;
      }
      const unsigned int o_excl = __shfl_sync(0xffffffffu, excl, own);
      const unsigned int o_rb = __shfl_sync(0xffffffffu, rb, own);
      const unsigned int o_v12 = __shfl_sync(0xffffffffu, v12, own);
      const unsigned int o_vp = __shfl_sync(0xffffffffu, vtp, own) >> 16;
      const unsigned long long o_sg0 = __shfl_sync(0xffffffffu, sg0, own);
      const unsigned long long o_sg1 = __shfl_sync(0xffffffffu, sg1, own);
      const unsigned int o_v1 = o_v12 & 0xFFFFu, o_v2 = o_v12 >> 16;
      bool is_child = false, exact = false;
      unsigned int v = 0;
      if (k < total) {
        v = ncol[o_rb + (k - o_excl)];
        if (v > o_v2 && v != o_vp) {
          const ulonglong2 ns = NS[v];
          const bool may_close = sig_test(ns.x, ns.y, sig_bit(o_v1));
          const bool may_chord = ((ns.x & o_sg0) | (ns.y & o_sg1)) != 0;
          if (!may_close && !may_chord) is_child = store;
          else exact = store || may_close;
        }
      }
      if (store) add_children(is_child, own, v);
      const unsigned int xb = __ballot_sync(0xffffffffu, exact);
      if (nexact + __popc(xb) > CX) run_exact();
      if (exact) sx[nexact + __popc(xb & lt_mask)] = own << 16 | v;
      nexact += __popc(xb);
      __syncwarp();
    }
    if (nexact) run_exact();
    if (nchild) flush();
    __syncwarp();
  }
  __shared__ unsigned long long s_red3[96];
  block_sum3_u64(ncyc, hacc, nbound, s_red3);
  if (threadIdx.x == 0) {
    if (ncyc) atomicAdd(&p.hist[t + 1], ncyc);
    if (hacc) atomicAdd(p.hash, hacc);
    if (nbound) atomicAdd(&p.ctl->nxt[s % 3], nbound);
  }
}

// The last level (t + 1 = L', or no room for children): nothing is stored, so only a
// closing candidate counts, and it neighbours both vt and v1.  The records stream through
// registers (the next group loaded while the current one is filtered, later ones
// prefetched into L2 by the bulk-copy engine); a path whose end vertices have disjoint
// neighbour signatures is finished after that one test.  The others are queued as staged
// rows, and every 32 queued paths are expanded together: flattened (path, candidate)
// pairs, v1's bit in nsig(v) first, then v1 in Adj(v) (sorted row) and, for a closing,
// the chord test of Adj(v) against the staged ids.
template <int CAP, int MAXCAP>
__device__ __forceinline__ void process_csr_last(const EngineParams& p, const StepPlan& pl,
                                                 const unsigned int* nrow, const unsigned short* ncol,
                                                 const unsigned long long* nsig, const unsigned long long* rtab) {
  constexpr int NP = CAP / 2, RS = NP + 1, NQ = CAP / 8;
  constexpr unsigned int CX = 64;
  CsrSmem<CAP>& sm = csr_smem<CAP, MAXCAP>();
  const unsigned int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned int lt_mask = (1u << lane) - 1u;
  unsigned int* sq = sm.path[wid];  // queued rows
  unsigned int* sx = sm.exact[wid];
  const unsigned int t = pl.t;
  const unsigned int nv = csr_rec_u16(t) / 8, nw = (t + 1) / 2;
  const unsigned int wv = (t - 1) >> 1, sv = ((t - 1) & 1) * 16;  // word and shift of vt
  const uint4* S = reinterpret_cast<const uint4*>(p.arena + pl.src_base);
  const ulonglong2* NS = reinterpret_cast<const ulonglong2*>(nsig);
  unsigned long long ncyc = 0, hacc = 0;
  const unsigned long long wstep = (unsigned long long)gridDim.x * (blockDim.x >> 5) * 32;
  unsigned long long w0 = pl.begin + ((unsigned long long)wid * gridDim.x + blockIdx.x) * 32;
  uint4 nx[NQ];
  auto fetch = [&](unsigned long long base) {
    const unsigned long long i = base + lane;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      nx[q] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
      if (i < pl.end && (unsigned)q < nv) nx[q] = __ldcg(S + i * nv + q);
    }
  };
  auto prefetch = [&](unsigned long long base) {
    if (lane == 0 && base < pl.end) {
      const unsigned long long k = min(32ull, pl.end - base);
      bulk_prefetch_l2(S + base * nv, (unsigned int)(k * nv * 16));
    }
  };
  auto put_row = [&](unsigned int slot) {
    unsigned int* row = sq + slot * RS;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      row[4 * q] = nx[q].x;
      row[4 * q + 1] = nx[q].y;
      row[4 * q + 2] = nx[q].z;
      row[4 * q + 3] = nx[q].w;
    }
  };
  // expand the first `count` queued paths
  auto expand = [&](unsigned int count) {
    __syncwarp();
    const unsigned int* row = sq + lane * RS;
    unsigned int v12 = 0xFFFF0000u, vtp = 0, rb = 0, cnt = 0;
    if (lane < count) {
      v12 = row[0];
      const unsigned int vt = rec_id(row, t - 1);
      vtp = vt | rec_id(row, t - 2) << 16;
      rb = nrow[vt];
      cnt = nrow[vt + 1] - rb;
    }
    unsigned int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    const unsigned int excl = incl - cnt, total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned int nexact = 0;
    auto run_exact = [&]() {
      for (unsigned int r0 = 0; r0 < nexact; r0 += 32) {
        const bool act = r0 + lane < nexact;
        const unsigned int e = act ? sx[r0 + lane] : 0u;
        const unsigned int own = e >> 16, v = e & 0xFFFFu;
        const unsigned int o_v12 = __shfl_sync(0xffffffffu, v12, own);
        const unsigned int o_vt = __shfl_sync(0xffffffffu, vtp, own) & 0xFFFFu;
        const unsigned int o_v1 = o_v12 & 0xFFFFu, o_v2 = o_v12 >> 16;
        const unsigned int* orow = sq + own * RS;
        if (act) {
          const unsigned int f0 = nrow[v], f1 = nrow[v + 1];
          unsigned int f = f0;
          while (f < f1 && ncol[f] < o_v1) ++f;
          bool close = f < f1 && ncol[f] == o_v1, chord = false;
          for (f = f0; close && !chord && f < f1; ++f) {
            const unsigned int w = ncol[f];
            if (w < o_v2 || w == o_vt || w == o_v1) continue;
            chord = on_path(orow, nw, w);
          }
          if (close && !chord) {
            ++ncyc;
            unsigned long long hs = rtab[v];
            for (unsigned int j = 0; j < t; ++j) hs += rtab[rec_id(orow, j)];
            hacc += mix64(hs + (unsigned long long)(t + 1) * kGamma);
            if (p.cyc_vert)
              emit_cycle(p, t + 1, [&](unsigned int j) -> unsigned int { return j < t ? rec_id(orow, j) : v; });
          }
        }
      }
      nexact = 0;
      __syncwarp();
    };
    for (unsigned int r0 = 0; r0 < total; r0 += 32) {
      const unsigned int k = r0 + lane;
      unsigned int own = 0;
#pragma unroll
      for (int b = 16; b >= 1; b >>= 1) {
        const unsigned int e = __shfl_sync(0xffffffffu, excl, (own + b) & 31);
        if (own + b < 32 && e <= k) own += b;
      }
      const unsigned int o_excl = __shfl_sync(0xffffffffu, excl, own);
      const unsigned int o_rb = __shfl_sync(0xffffffffu, rb, own);
      const unsigned int o_v12 = __shfl_sync(0xffffffffu, v12, own);
      const unsigned int o_vp = __shfl_sync(0xffffffffu, vtp, own) >> 16;
      bool exact = false;
      unsigned int v = 0;
      if (k < total) {
        v = ncol[o_rb + (k - o_excl)];
        if (v > (o_v12 >> 16) && v != o_vp) {
          const ulonglong2 ns = NS[v];
          exact = sig_test(ns.x, ns.y, sig_bit(o_v12 & 0xFFFFu));
        }
      }
      const unsigned int xb = __ballot_sync(0xffffffffu, exact);
      if (nexact + __popc(xb) > CX) run_exact();
      if (exact) sx[nexact + __popc(xb & lt_mask)] = own << 16 | v;
      nexact += __popc(xb);
      __syncwarp();
    }
    if (nexact) run_exact();
    __syncwarp();
  };

  unsigned int qn = 0;  // queued paths (the same in every lane)
  if (w0 < pl.end) fetch(w0);
#pragma unroll
  for (int d = 1; d <= 4; ++d) prefetch(w0 + d * wstep);
  for (; w0 < pl.end; w0 += wstep) {
    prefetch(w0 + 5 * wstep);
    bool surv = false;
    if (w0 + lane < pl.end) {
      unsigned int xt = 0;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        if ((unsigned)(4 * q) == wv) xt = nx[q].x;
        if ((unsigned)(4 * q + 1) == wv) xt = nx[q].y;
        if ((unsigned)(4 * q + 2) == wv) xt = nx[q].z;
        if ((unsigned)(4 * q + 3) == wv) xt = nx[q].w;
      }
      const unsigned int v1 = nx[0].x & 0xFFFFu, vt = (xt >> sv) & 0xFFFFu;
      const ulonglong2 a = NS[vt], c = NS[v1];
      surv = ((a.x & c.x) | (a.y & c.y)) != 0;
    }
    const unsigned int bal = __ballot_sync(0xffffffffu, surv);
    const unsigned int ns = __popc(bal), rank = __popc(bal & lt_mask);
    const unsigned int take = min(ns, 32u - qn);
    if (surv && rank < take) put_row(qn + rank);
    if (qn + ns >= 32) {
      expand(32);
      __syncwarp();
      if (surv && rank >= take) put_row(rank - take);
      qn = ns - take;
    } else {
      qn += ns;
    }
    __syncwarp();
    if (w0 + wstep < pl.end) fetch(w0 + wstep);
  }
  if (qn) expand(qn);
  __shared__ unsigned long long s_red4[96];
  unsigned long long zero = 0;
  block_sum3_u64(ncyc, hacc, zero, s_red4);
  if (threadIdx.x == 0) {
    if (ncyc) atomicAdd(&p.hist[t + 1], ncyc);
    if (hacc) atomicAdd(p.hash, hacc);
  }
}

// Set the u16 at position e (0..7) of a 16-byte chunk of ids.
__device__ __forceinline__ void chunk_set_u16(uint4& c, unsigned int e, unsigned int v) {
  const unsigned int sh = (e & 1u) * 16u, m = 0xFFFFu << sh, x = (v & 0xFFFFu) << sh;
  switch (e >> 1) {
    case 0: c.x = (c.x & ~m) | x; break;
    case 1: c.y = (c.y & ~m) | x; break;
    case 2: c.z = (c.z & ~m) | x; break;
    default: c.w = (c.w & ~m) | x; break;
  }
}

// True if any u16 of the chunk equals w (a zero 16-bit lane of c ^ ww marks an equal id).
__device__ __forceinline__ bool chunk_has_u16(const uint4& c, unsigned int ww) {
  auto z = [](unsigned int x) { return (x - 0x00010001u) & ~x & 0x80008000u; };
  return (z(c.x ^ ww) | z(c.y ^ ww) | z(c.z ^ ww) | z(c.w ^ ww)) != 0u;
}

// Candidates with more neighbours than this are tested against the path by looking the
// path up in their row, not by listing their neighbours as queries.
constexpr unsigned int kLongQueryMaxDeg = 32;

// True if the sorted row holds x (binary search).
__device__ __forceinline__ bool row_has(const unsigned short* row, unsigned int d, unsigned int x) {
  unsigned int lo = 0, hi = d;
  while (lo < hi) {
    const unsigned int mid = (lo + hi) >> 1, y = row[mid];
    if (y == x) return true;
    if (y < x) lo = mid + 1;
    else hi = mid;
  }
  return false;
}

// The same expansion for paths of more than 64 vertices, one warp per path.  The record
// is read in coalesced 16-byte chunks (lane l takes chunks l, l + 32, ...).  A round takes
// up to 32 candidates v in Adj(vt) (one per lane, label test and v != v_{t-1}).  A
// candidate of low degree lists its neighbours w >= v2 other than vt and v1 as queries
// ("is w an interior vertex?"), and one pass of the warp over the record answers every
// query of the round (queries in shared memory, hits OR-reduced over the lanes).  A
// candidate of high degree is tested the other way round: every interior vertex is
// looked up in its sorted row (binary search, the warp's lanes over the record), and v1
// too.  A candidate without a chord closes a cycle if v1 is its neighbour (hash: the
// path's r-sum, a warp sum, plus r(v)), and is otherwise a child, copied chunk by chunk
// with its id appended.
__device__ __forceinline__ void process_csr_long_warp(const EngineParams& p, const StepPlan& pl,
                                                      const unsigned int* nrow, const unsigned short* ncol,
                                                      const unsigned long long* nsig, const unsigned long long* rtab,
                                                      unsigned long long* s_red) {
  constexpr unsigned int QC = 32;  // queries per pass
  __shared__ unsigned int s_q[kMaxThreads / 32][QC];
  __shared__ unsigned char s_own[kMaxThreads / 32][QC];
  const unsigned int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned int* sq = s_q[wid];
  unsigned char* so = s_own[wid];
  const unsigned int t = pl.t, L = p.L;
  const unsigned int R = csr_rec_u16(t), R2 = csr_rec_u16(t + 1), NC = R / 8, NC2 = R2 / 8;
  const unsigned short* S = reinterpret_cast<const unsigned short*>(p.arena + pl.src_base);
  unsigned short* D = reinterpret_cast<unsigned short*>(p.arena + pl.dst_base);
  const unsigned long long ds = pl.dst_stride;
  const bool store = ds != 0;
  const bool close_ok = t + 1 <= L, bound_ok = t + 2 < L;
  const unsigned long long s = pl.s;
  const unsigned long long gam = (unsigned long long)(t + 1) * kGamma;
  unsigned long long ncyc = 0, hacc = 0, nbound = 0;
  const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  // warp w of block b takes the (w * gridDim + b)-th path, so the warps of a small level
  // land on different SMs
  const unsigned long long gw = (unsigned long long)wid * gridDim.x + blockIdx.x;
  for (unsigned long long i = pl.begin + gw; i < pl.end; i += nw) {  // warp-uniform
    const unsigned short* rec = S + i * R;
    const uint4* rc = reinterpret_cast<const uint4*>(rec);
    const unsigned int v1 = ldcg16(rec), v2 = ldcg16(rec + 1), vp = ldcg16(rec + t - 2), vt = ldcg16(rec + t - 1);
    const unsigned int rb = nrow[vt], deg = nrow[vt + 1] - rb;
    bool have_h = false;
    unsigned long long hsum = 0;
    for (unsigned int c0 = 0; c0 < deg; c0 += 32) {
      const unsigned int q = c0 + lane;
      const unsigned int v = q < deg ? (unsigned int)ncol[rb + q] : 0xFFFFFFFFu;
      const bool cand = q < deg && v > v2 && v != vp;
      // this candidate's queries
      bool close = false;
      unsigned int nq = 0, eb = 0, ee = 0;
      if (cand) {
        eb = nrow[v];
        ee = nrow[v + 1];
      }
      const bool big = cand && ee - eb > kLongQueryMaxDeg;
      if (cand && !big) {
        for (unsigned int e = eb; e < ee; ++e) {
          const unsigned int w = ncol[e];
          if (w < v2 || w == vt) continue;
          if (w == v1) close = true;
          else ++nq;
        }
      }
      unsigned int incl = nq;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += y;
      }
      const unsigned int off = incl - nq, qtot = __shfl_sync(0xffffffffu, incl, 31);
      bool chord = false;
      for (unsigned int q0 = 0; q0 < qtot; q0 += QC) {
        if (nq && off < q0 + QC && off + nq > q0) {
          unsigned int k = off;
          for (unsigned int e = eb; e < ee; ++e) {
            const unsigned int w = ncol[e];
            if (w < v2 || w == vt || w == v1) continue;
            if (k >= q0 && k < q0 + QC) {
              sq[k - q0] = w;
              so[k - q0] = (unsigned char)lane;
            }
            ++k;
          }
        }
        __syncwarp();
        const unsigned int nqc = min(QC, qtot - q0);
        unsigned int hit = 0;
        for (unsigned int c = lane; c < NC; c += 32) {
          const uint4 x = __ldcg(rc + c);
          for (unsigned int qq = 0; qq < nqc; ++qq) {
            const unsigned int w = sq[qq];
            if (chunk_has_u16(x, w | (w << 16))) hit |= 1u << qq;
          }
        }
        hit = __reduce_or_sync(0xffffffffu, hit);
        while (hit) {
          const unsigned int qq = __ffs(hit) - 1;
          hit &= hit - 1;
          if (so[qq] == lane) chord = true;
        }
        __syncwarp();
      }
      // high-degree candidates, one at a time: interior vertices looked up in the row
      unsigned int bm = __ballot_sync(0xffffffffu, big);
      while (bm) {
        const unsigned int src = __ffs(bm) - 1;
        bm &= bm - 1;
        const unsigned int bb = __shfl_sync(0xffffffffu, eb, src), bd = __shfl_sync(0xffffffffu, ee, src) - bb;
        const unsigned short* row = ncol + bb;
        bool found = false;
        for (unsigned int c = lane; c < NC && !found; c += 32) {
          const uint4 x = __ldcg(rc + c);
          const unsigned int u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const unsigned int pos = 8u * c + k;
            if (pos >= 1 && pos + 1 < t && row_has(row, bd, (u[k >> 1] >> (16 * (k & 1))) & 0xFFFFu)) found = true;
          }
        }
        const bool any = __any_sync(0xffffffffu, found);
        if (lane == src) {
          chord = any;
          close = row_has(row, bd, v1);
        }
      }
      const bool closes = cand && !chord && close;
      const bool child = cand && !chord && !close && store;
      if (close_ok && __any_sync(0xffffffffu, closes)) {
        if (!have_h) {  // the path's r-sum, once per path
          unsigned long long h = 0;
          for (unsigned int c = lane; c < NC; c += 32) {
            const uint4 x = __ldcg(rc + c);
            const unsigned int u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (8u * c + k < t) h += rtab[(u[k >> 1] >> (16 * (k & 1))) & 0xFFFFu];
          }
          hsum = warp_sum_u64(h);
          have_h = true;
        }
        if (closes) {
          ++ncyc;
          hacc += mix64(hsum + rtab[v] + gam);
          if (p.cyc_vert)
            emit_cycle(p, t + 1, [&](unsigned int j) -> unsigned int {
              return j < t ? (unsigned int)ldcg16(rec + j) : v;
            });
        }
      }
      const unsigned int cm = __ballot_sync(0xffffffffu, child);
      if (cm == 0) continue;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(&p.ctl->cnt[s % 3], (unsigned long long)__popc(cm));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (child && bound_ok) nbound += nrow[v + 1] - nrow[v] - 1;
      if (p.cyc_stream && t + 2 <= L) {  // streamed lists: the children's closing bound
        const unsigned int k = __reduce_add_sync(0xffffffffu, child ? closing_bound(nrow, ncol, nsig, v, v1, vt) : 0u);
        if (lane == 0 && k) atomicAdd(&p.ctl->ncl[s % 3], (unsigned long long)k);
      }
      unsigned int rest = cm;
      for (unsigned long long slot = base; rest; ++slot) {  // one child at a time, warp-wide copy
        const unsigned int src = __ffs(rest) - 1;
        rest &= rest - 1;
        const unsigned int cv = __shfl_sync(0xffffffffu, v, src);
        if (slot < ds) {
          uint4* out = reinterpret_cast<uint4*>(D + slot * R2);
          for (unsigned int c = lane; c < NC2; c += 32) {
            uint4 x = c < NC ? __ldcg(rc + c) : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
            if (c == t / 8) chunk_set_u16(x, t % 8, cv);
            out[c] = x;
          }
        } else if (lane == 0) {
          set_err(p.ctl, kDevBounds, 2);
        }
      }
    }
  }
  block_sum3_u64(ncyc, hacc, nbound, s_red);
  if (threadIdx.x == 0) {
    if (ncyc) atomicAdd(&p.hist[t + 1], ncyc);
    if (hacc) atomicAdd(p.hash, hacc);
    if (nbound) atomicAdd(&p.ctl->nxt[s % 3], nbound);
  }

}

// ------------------------------------------------------------------ the persistent kernel

// Hardware barrier of a thread-block cluster (all threads of all CTAs of the cluster),
// with release/acquire ordering of global and shared memory at cluster scope.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// NT threads per block.  NT = 256: the persistent grid (cooperative launch, grid barrier).
// NT = 1024: the small phase, one thread-block cluster whose steps are separated by the
// hardware cluster barrier; it runs while the frames are small (p.handover) and leaves
// the state for the grid launch that follows.  Every CTA computes the same plan, so all
// CTAs of the cluster execute the same sequence of cluster barriers.
template <Kind K, int NT>
__global__ void __launch_bounds__(NT, NT >= 1024 ? 1 : KindTraits<K>::minB) engine_kernel(EngineParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ StepPlan pl;
  __shared__ LocalState st;
  __shared__ unsigned int s_warp[NT / 32 + 1];
  __shared__ unsigned long long s_red[96];
  __shared__ unsigned long long s_base;
  __shared__ __align__(8) unsigned long long s_mbar;
  const unsigned int tid = threadIdx.x;

  const unsigned long long* adj = p.adj;
  const unsigned long long* rtab = p.rtab;
  const unsigned int* nrow = p.nrow;
  const unsigned short* ncol = p.ncol;
  const unsigned long long* nsig = p.nsig;
  if (p.smem_graph) {
    // stage the relabelled graph into shared memory with the bulk-copy (TMA) engine:
    // bitset rows + r-table, or CSR rows + neighbours + neighbour signatures
    if (tid == 0) mbar_init(&s_mbar, 1);
    __syncthreads();
    if (tid == 0) {
      if constexpr (KindTraits<K>::csr) {
        mbar_arrive_expect_tx(&s_mbar, p.adj_bytes + p.nsig_bytes);
        bulk_copy_g2s(smem, p.nrow, p.row_bytes, &s_mbar);
        bulk_copy_g2s(smem + p.row_bytes, p.ncol, p.adj_bytes - p.row_bytes, &s_mbar);
        bulk_copy_g2s(smem + p.adj_bytes, p.nsig, p.nsig_bytes, &s_mbar);
      } else {
        mbar_arrive_expect_tx(&s_mbar, p.adj_bytes + p.rtab_bytes);
        bulk_copy_g2s(smem, p.adj, p.adj_bytes, &s_mbar);
        bulk_copy_g2s(smem + p.adj_bytes, p.rtab, p.rtab_bytes, &s_mbar);
      }
    }
    unsigned int polls = 0;
    while (!mbar_try_wait(&s_mbar, 0)) {
      if (++polls > (1u << 22)) {
        set_err(p.ctl, kDevTimeout, 2);
        break;
      }
    }
    if constexpr (KindTraits<K>::csr) {
      nrow = reinterpret_cast<const unsigned int*>(smem);
      ncol = reinterpret_cast<const unsigned short*>(smem + p.row_bytes);
      nsig = reinterpret_cast<const unsigned long long*>(smem + p.adj_bytes);
    } else {
      adj = reinterpret_cast<const unsigned long long*>(smem);
      rtab = reinterpret_cast<const unsigned long long*>(smem + p.adj_bytes);
    }
  }

  // Step counters (child slots, next-level size): global for the persistent grid; in the
  // cluster phase they live in CTA 0's shared memory and every CTA reaches them as
  // distributed shared memory (no L2 round trip for the slot atomics and the reads)
  __shared__ unsigned long long s_ctr[6];
  unsigned long long* cntp = p.ctl->cnt;
  unsigned long long* nxtp = p.ctl->nxt;
  if constexpr (NT >= 1024) {
    if (tid < 6) s_ctr[tid] = 0ull;
    unsigned long long* c0 = cooperative_groups::this_cluster().map_shared_rank(s_ctr, 0);
    cntp = c0;
    nxtp = c0 + 3;
    cluster_barrier();  // the zeros are visible before any CTA adds to them
  }

  if (tid == 0) {
    Control* c = p.ctl;
    if (p.fresh) {
      const unsigned long long n0 = c->seed_count;
      st.depth = n0 ? 1u : 0u;
      st.bot = n0 ? p.seed_bytes : 0ull;
      st.top = p.arena_bytes;
      st.cur.base = 0;
      st.cur.bytes = p.seed_bytes;
      st.cur.stride = p.seed_stride;
      st.cur.count = n0;
      st.cur.cursor = 0;
      st.cur.next = c->seed_next;
      st.cur.ncl = kNoNext;
      st.cur.t = KindTraits<K>::multi ? 0u : 3u;
      st.cur.end = 0;
      if (blockIdx.x == 0) c->t_start = globaltimer();
      if (blockIdx.x == 0 && n0) store_frame(&p.frames[0], st.cur);
      if (n0 && p.seed_bytes > c->peak) c->peak = p.seed_bytes;
    } else {
      st.depth = c->depth;
      st.bot = c->bot;
      st.top = c->top;
      if (st.depth) st.cur = load_frame(&p.frames[st.depth - 1]);
    }
    pl.s = c->step;
    st.gen = ld_acquire_u32(&c->bar_gen);
    st.peak = c->peak;
    // an error already raised (by seeding) stops the expansion before its first step
    if (ld_relaxed_i32(&c->err) != 0) st.depth = 0;
  }
  __syncthreads();
  unsigned long long s = pl.s;
  unsigned int steps_here = 0;
  for (;;) {
    if (tid == 0) {
      bool go = p.max_steps == 0 || steps_here < p.max_steps;
      if (go) go = plan_step<K>(p, st, pl);
      // small phase: stop before a level that is too large for one cluster (the plan has
      // only popped finished frames, which the state written back below keeps)
      if (go && p.handover && pl.end - pl.begin > p.handover) go = false;
      pl.done = go ? 0u : 1u;
      pl.s = s;
    }
    __syncthreads();
    if (pl.done) break;
    if constexpr (KindTraits<K>::csr) {
      constexpr int CAP = KindTraits<K>::cap;  // ids a staged row holds: 16, 32 or 64
      constexpr int C32 = CAP >= 32 ? 32 : 16, C64 = CAP >= 64 ? 64 : 16;
      if (pl.dst_stride == 0 && pl.t <= 16) process_csr_last<16, CAP>(p, pl, nrow, ncol, nsig, rtab);
      else if (pl.dst_stride == 0 && CAP >= 32 && pl.t <= 32) process_csr_last<C32, CAP>(p, pl, nrow, ncol, nsig, rtab);
      else if (pl.dst_stride == 0 && CAP >= 64 && pl.t <= 64) process_csr_last<C64, CAP>(p, pl, nrow, ncol, nsig, rtab);
      else if (pl.t <= 16) process_csr_coop<16, CAP>(p, pl, nrow, ncol, nsig, rtab);
      else if (CAP >= 32 && pl.t <= 32) process_csr_coop<C32, CAP>(p, pl, nrow, ncol, nsig, rtab);
      else if (CAP >= 64 && pl.t <= 64) process_csr_coop<C64, CAP>(p, pl, nrow, ncol, nsig, rtab);
      else process_csr_long_warp(p, pl, nrow, ncol, nsig, rtab, s_red);
    } else {
      // the flattened form for the persistent grid (the small cluster phase keeps the
      // per-lane forms: its levels are small and its 32 warps per block would need 4x the
      // staging memory)
      if constexpr (NT >= 1024) {
        if constexpr (KindTraits<K>::W <= kFuseLaneMaxW) {
          if (pl.fuse) process_bitset_fused_lane<K>(p, pl, adj, rtab, s_red, cntp, nxtp);
          else process_bitset<K>(p, pl, adj, rtab, s_warp, s_red, &s_base, cntp, nxtp);
        } else {
          process_bitset<K>(p, pl, adj, rtab, s_warp, s_red, &s_base, cntp, nxtp);
        }
      }
      else if constexpr (KindTraits<K>::multi) process_multi_flat<NT>(p, pl, adj, rtab);
      else if (pl.fuse) process_bitset_fused<K, NT>(p, pl, adj, rtab, s_red);
      else process_bitset_flat<K, NT>(p, pl, adj, rtab, s_red);
    }
    if (blockIdx.x == 0 && tid == 0) {
      cntp[(s + 1) % 3] = 0;
      nxtp[(s + 1) % 3] = 0;
      p.ctl->take[(s + 1) % 3] = 0;
      if (p.cyc_stream) p.ctl->ncl[(s + 1) % 3] = 0;
    }
    if (p.cluster) {
      cluster_barrier();
    } else if (!grid_barrier(p.ctl, gridDim.x, p.spin_limit, st.gen)) {
      break;
    }
    if (tid == 0) {
      // the step's counters and the error word, in one round trip
      unsigned long long c, nx;
      if constexpr (NT >= 1024) {
        c = *reinterpret_cast<volatile unsigned long long*>(&cntp[s % 3]);
        nx = *reinterpret_cast<volatile unsigned long long*>(&nxtp[s % 3]);
      } else {
        c = ld_relaxed_u64(&p.ctl->cnt[s % 3]);
        nx = ld_relaxed_u64(&p.ctl->nxt[s % 3]);
      }
      // (the cluster phase has no barrier that can time out and a child count is clamped to
      // its frame, so it leaves the error word to the grid phase and to the host)
      const int err = NT >= 1024 ? 0 : ld_relaxed_i32(&p.ctl->err);
      const unsigned long long ncl = p.cyc_stream ? ld_relaxed_u64(&p.ctl->ncl[s % 3]) : kNoNext;
      commit_step<K>(p, st, c, nx, ncl, blockIdx.x == 0);
      if (err != 0) st.depth = 0;  // every block reads the same word: all stop here
      if (blockIdx.x == 0 && p.step_ts && s < p.step_ts_cap) {
        p.step_ts[s] = globaltimer();
        if (p.step_rec) p.step_rec[s] = st.expanded;
      }
    }
    ++s;
    ++steps_here;
  }
  // cluster phase: CTA 0's shared memory (the counters) must outlive every CTA's reads
  if constexpr (NT >= 1024) cluster_barrier();
  if (blockIdx.x == 0 && tid == 0) {
    Control* c = p.ctl;
    c->depth = st.depth;
    c->bot = st.bot;
    c->top = st.top;
    if (st.depth) store_frame(&p.frames[st.depth - 1], st.cur);
    c->step = s;
    c->peak = st.peak;
  }
}

// ------------------------------------------------------------------ host-side launch helpers

static const void* engine_fn(Kind k) {
  switch (k) {
    case Kind::Bitset1: return (const void*)engine_kernel<Kind::Bitset1, kMaxThreads>;
    case Kind::Bitset2: return (const void*)engine_kernel<Kind::Bitset2, kMaxThreads>;
    case Kind::Bitset4: return (const void*)engine_kernel<Kind::Bitset4, kMaxThreads>;
    case Kind::Multi: return (const void*)engine_kernel<Kind::Multi, kMaxThreads>;
    case Kind::Csr: return (const void*)engine_kernel<Kind::Csr, kMaxThreads>;
    case Kind::Csr16: return (const void*)engine_kernel<Kind::Csr16, kMaxThreads>;
    case Kind::Csr32: return (const void*)engine_kernel<Kind::Csr32, kMaxThreads>;
  }
  return nullptr;
}

static const void* small_engine_fn(Kind k) {
  switch (k) {
    case Kind::Bitset1: return (const void*)engine_kernel<Kind::Bitset1, kSmallThreads>;
    case Kind::Bitset2: return (const void*)engine_kernel<Kind::Bitset2, kSmallThreads>;
    case Kind::Bitset4: return (const void*)engine_kernel<Kind::Bitset4, kSmallThreads>;
    default: return nullptr;
  }
}

// The dynamic shared memory limit of a kernel is only ever raised.  A captured CUDA graph
// keeps each kernel node's shared memory size but not the function attribute, so lowering
// the attribute for a later launch of a smaller graph would make a replayed node of a
// larger graph ask for more than its function allows.
static std::mutex g_smem_mutex;
static std::vector<std::pair<const void*, size_t>> g_smem_set;

static cudaError_t allow_smem(const void* fn, size_t smem) {
  std::lock_guard<std::mutex> lock(g_smem_mutex);
  for (auto& kv : g_smem_set)
    if (kv.first == fn) {
      if (kv.second >= smem) return cudaSuccess;
      const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) kv.second = smem;
      return e;
    }
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) g_smem_set.push_back({fn, smem});
  return e;
}

cudaError_t engine_occupancy(Kind kind, int block, size_t smem, int* blocks_per_sm) {
  const void* fn = engine_fn(kind);
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

cudaError_t launch_engine(Kind kind, const EngineParams& p, int grid, int block, size_t smem, cudaStream_t st) {
  const void* fn = engine_fn(kind);
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  EngineParams copy = p;
  copy.cluster = 0;
  copy.handover = 0;
  void* args[] = {(void*)&copy};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

// Largest usable cluster (at most 16 CTAs of kSmallThreads threads), 0 if clusters of this
// kernel cannot be launched (then the small phase is skipped).
int small_cluster_size(Kind kind, size_t smem) {
  const void* fn = small_engine_fn(kind);
  if (!fn) return 0;
  if (allow_smem(fn, smem) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(kSmallThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = 16;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int cs = 0;
  if (cudaOccupancyMaxPotentialClusterSize(&cs, fn, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return cs >= 16 ? 16 : (cs >= 8 ? 8 : 0);
}

cudaError_t launch_small_engine(Kind kind, const EngineParams& p, int cluster, size_t smem,
                                unsigned long long handover, cudaStream_t st) {
  const void* fn = small_engine_fn(kind);
  if (!fn || cluster <= 0) return cudaErrorInvalidValue;
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  EngineParams copy = p;
  copy.cluster = 1;
  copy.handover = handover;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(kSmallThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = cluster;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  void* args[] = {(void*)&copy};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace cc
