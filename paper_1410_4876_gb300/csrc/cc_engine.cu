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
// adjacency) and process_bitset / process_bitset_fused_lane (the small-level cluster
// phase) in cc_expand_bitset.cuh; process_multi_flat (batch and serving) in
// cc_expand_multi.cuh; process_csr_coop / process_csr_last / process_csr_long_warp (CSR
// adjacency) in cc_expand_csr.cuh.
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
  static constexpr int PF = K == Kind::Bitset1 ? 4 : (K == Kind::Bitset2 ? 2 : 1);
  // children staged per batch in a two-level step, in rounds of 32 (shared memory bound)
  static constexpr int PF2 = K == Kind::Bitset1 ? 4 : 1;
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

// ------------------------------------------------------------------ expansion forms

#include "cc_expand_bitset.cuh"
#include "cc_expand_multi.cuh"
#include "cc_expand_csr.cuh"

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
// SG: the graph is staged in shared memory (known at compile time, so the expansion's graph
// reads are shared-memory loads): always for one graph's bitset rows (n <= 256: at most 10 KB
// with the r-table), never for the batch, and for CSR graphs whose rows fit.
template <Kind K, int NT, bool SG>
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
  if constexpr (SG) {
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
    } else if constexpr (KindTraits<K>::W == 1) {
      adj = reinterpret_cast<const unsigned long long*>(smem);
      rtab = reinterpret_cast<const unsigned long long*>(smem + p.adj_bytes);
    } else {
      // wider rows keep generic loads (selected at run time): measured faster for them
      // (grid 8x10: 37.4 against 45.5 ms with shared-memory loads known at compile time)
      adj = p.smem_graph ? reinterpret_cast<const unsigned long long*>(smem) : p.adj;
      rtab = p.smem_graph ? reinterpret_cast<const unsigned long long*>(smem + p.adj_bytes) : p.rtab;
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

// `staged`: the launch stages the graph in shared memory (p.smem_graph; a CSR graph whose
// rows fit); one graph's bitset rows always are, the batch's never.
static const void* engine_fn(Kind k, bool staged) {
  switch (k) {
    case Kind::Bitset1: return (const void*)engine_kernel<Kind::Bitset1, kMaxThreads, true>;
    case Kind::Bitset2: return (const void*)engine_kernel<Kind::Bitset2, kMaxThreads, true>;
    case Kind::Bitset4: return (const void*)engine_kernel<Kind::Bitset4, kMaxThreads, true>;
    case Kind::Multi: return (const void*)engine_kernel<Kind::Multi, kMaxThreads, false>;
    case Kind::Csr:
      return staged ? (const void*)engine_kernel<Kind::Csr, kMaxThreads, true>
                    : (const void*)engine_kernel<Kind::Csr, kMaxThreads, false>;
    case Kind::Csr16:
      return staged ? (const void*)engine_kernel<Kind::Csr16, kMaxThreads, true>
                    : (const void*)engine_kernel<Kind::Csr16, kMaxThreads, false>;
    case Kind::Csr32:
      return staged ? (const void*)engine_kernel<Kind::Csr32, kMaxThreads, true>
                    : (const void*)engine_kernel<Kind::Csr32, kMaxThreads, false>;
  }
  return nullptr;
}

static const void* small_engine_fn(Kind k) {
  switch (k) {
    case Kind::Bitset1: return (const void*)engine_kernel<Kind::Bitset1, kSmallThreads, true>;
    case Kind::Bitset2: return (const void*)engine_kernel<Kind::Bitset2, kSmallThreads, true>;
    case Kind::Bitset4: return (const void*)engine_kernel<Kind::Bitset4, kSmallThreads, true>;
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
  const void* fn = engine_fn(kind, smem > 0);
  cudaError_t e = allow_smem(fn, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

cudaError_t launch_engine(Kind kind, const EngineParams& p, int grid, int block, size_t smem, cudaStream_t st) {
  const void* fn = engine_fn(kind, p.smem_graph != 0);
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
