// Internal device/host definitions of the chordless-cycle library (sm_103a).
//
// Frontier layout.  Chordless paths in flight live in one device arena used as two
// stacks that grow towards each other (bottom end upwards, top end downwards).  A
// "frame" is a set of paths stored as structure-of-arrays planes inside one region;
// expanding (part of) a frame writes the children into a new region at the OTHER end.
// When every level fits, this is a ping-pong between the two ends, i.e. the
// level-synchronous T -> T' step of Algorithm 3 / Algorithm 4 (Section 4.4).  When a level
// would not fit, the frame is expanded in chunks and each chunk's subtree is finished
// depth-first before the next chunk (bounded frontier).
//
// Record formats (one path per record):
//   bitset, one graph, W = ceil(n/64) words:  B[W] (u64 planes), H (u64), M (u32)
//       B  blocked set: union of Adj(v_i) over the interior v_2..v_{t-1}, plus every
//          vertex whose label is <= l(v_2).  A candidate v of Adj(v_t) passes the label
//          test and the chord test of Algorithm 3 iff v is not in B.
//       H  sum of r(original id) over the path's vertices (running cycle-hash input).
//       M  v_1 | v_t << 16 (relabelled ids).
//   bitset, many graphs (n <= 64, W = 1): same planes, M = v1 | vt<<6 | t<<12 | slot<<18,
//       and N (u8): the path's exact number of children (0 when they would reach L').
//   CSR, one graph: one record per path, its relabelled u16 ids in order padded with 0xFFFF
//       to a multiple of 8 ids (16-byte vector accesses).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cc {

constexpr unsigned long long kGamma = 0x9E3779B97F4A7C15ull;

// SplitMix64 output finaliser (Steele, Lea and Flood 2014; constants of Vigna's
// public-domain splitmix64.c).  Device twin of the definition stated in cc.h.
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ unsigned long long vertex_r(unsigned int v) {
  return mix64((unsigned long long)(v + 1ull) * kGamma);
}

// Neighbour signatures of the CSR expansion: vertex x (relabelled id) stands for bit
// sig_bit(x) of a 128-bit word pair (Knuth's multiplicative hash, top 7 bits).  nsig(v) is
// the OR over Adj(v); a path's interior signature is the OR over v2..v_{t-1}.  Disjoint
// signatures prove that no neighbour of v lies on the interior (no chord); a set bit only
// means "maybe", and the exact test decides.
__host__ __device__ __forceinline__ unsigned int sig_bit(unsigned int x) { return (x * 2654435761u) >> 25; }

// Device error words (Control::err).
enum : int {
  kDevOk = 0,
  kDevTimeout = 1,   // a grid barrier or an mbarrier wait hit its poll limit
  kDevCapacity = 2,  // frontier arena too small to expand even one path
  kDevBounds = 3,    // a write would leave its region (self-check; skipped, never done)
  kDevDepth = 4,     // frame chain deeper than its array
  kDevSeedCap = 5,   // initial triplets exceeded their region
};

constexpr unsigned long long kNoNext = ~0ull;
constexpr int kMultiMaxN = 64;        // batch graphs: n <= 64, one u64 adjacency row
constexpr int kMultiHistStride = 65;  // lengths 0..64
constexpr unsigned kMultiMaxSlots = 1u << 14;
constexpr unsigned kBitsetMaxN = 256;
constexpr unsigned kCsrMaxN = 32768;

struct Frame {
  unsigned long long base;    // byte offset of the region in the arena
  unsigned long long bytes;   // region size
  unsigned long long stride;  // records per plane
  unsigned long long count;   // records present
  unsigned long long cursor;  // records already expanded
  unsigned long long next;    // exact number of children of the whole frame, or kNoNext
  unsigned long long ncl;     // streamed CSR lists: bound on the frame's closings, or kNoNext
  unsigned int t;             // path length (one-graph modes); 0 = per record (batch)
  unsigned int end;           // 0 = bottom stack, 1 = top stack
};

constexpr unsigned int kBarGroupSize = 16;  // blocks per first-level barrier counter
constexpr unsigned int kBarGroupPad = 8;    // one 32-byte sector per group counter
constexpr unsigned int kMaxBarGroups = 256;

// The words that many blocks touch at once each sit on their own 128-byte line: the
// per-step counters (atomics from every warp), the barrier generation and error word
// (polled by waiting blocks) and the grid-level arrival counter.
struct Control {
  alignas(128) unsigned long long cnt[3];  // children written in step s (index s % 3)
  unsigned long long nxt[3];               // children-of-children of step s (next frame size)
  unsigned long long ncl[3];               // streamed CSR lists: closing bound of step s's children
  alignas(128) unsigned long long take[3]; // batch: records of step s handed out to warps so far
  alignas(128) unsigned int bar_gen;       // barrier generation (released by the last group)
  int err;                                 // first device error (kDev*), 0 if none
  int err_info;
  alignas(128) unsigned int bar_count;     // groups arrived at the current grid barrier
  alignas(128) unsigned int bar_group[kMaxBarGroups * kBarGroupPad];  // blocks arrived, per group
  unsigned long long step;   // global step counter (continues across launches)
  unsigned long long bot;    // bottom stack top (bytes)
  unsigned long long top;    // top stack bottom (bytes)
  unsigned long long peak;   // largest extent in use (bytes)
  unsigned int depth;        // frames in the chain
  unsigned int spilled;      // a frame was expanded in more than one chunk
  unsigned long long seed_count;  // initial triplets (set by the seed kernel)
  unsigned long long seed_next;   // their children (exact)
  unsigned long long cyc_count;   // cycles offered to the cycle list
  unsigned long long cyc_verts;   // vertices offered to the cycle list
  unsigned long long t_start;     // globaltimer when a fresh engine launch started
  unsigned int want_offload;      // host frontier: the engine stopped to have frames moved to host memory
};

// Engine variants.  Csr16/Csr32 keep paths of up to 16/32 vertices in registers (chosen
// from L'); Csr handles any length (paths up to 64 vertices in registers, longer ones
// re-read from the frontier).
enum class Kind : int { Bitset1 = 0, Bitset2 = 1, Bitset4 = 2, Multi = 3, Csr = 4, Csr16 = 5, Csr32 = 6 };
__host__ __device__ constexpr bool is_csr(Kind k) { return k == Kind::Csr || k == Kind::Csr16 || k == Kind::Csr32; }

struct EngineParams {
  unsigned char* arena;
  unsigned long long arena_bytes;
  Control* ctl;
  Frame* frames;
  unsigned int max_depth;
  unsigned int n;        // one graph: vertices
  unsigned int L;        // one graph: L'
  unsigned int maxch;    // bound on children per path (max degree - 1, at least 1)
  const unsigned long long* adj;   // bitset rows, relabelled (one graph: n*W; batch: slot*64)
  const unsigned long long* rtab;  // r(original id) by relabelled id (one graph: n; batch: slot*64)
  const unsigned int* nrow;        // CSR (one graph): relabelled row offsets [n+1]
  const unsigned short* ncol;      // CSR: relabelled sorted neighbours
  unsigned char* Lg;               // batch: L' per slot
  const unsigned int* perm;        // one graph: relabelled id -> original id
  unsigned long long* hist;        // one graph: [L+1]; batch: [slot*65 + k]
  unsigned long long* hash;        // one graph: [1]; batch: [slot]
  unsigned long long* tcount;      // one graph: [L+1]; batch: [slot*65 + t]
  unsigned int* last_step;         // batch: 1 + the last step that expanded a path of the slot (0: none)
  long long* live;                 // batch/serving: paths of the slot still in flight
  unsigned long long* step_ts;     // globaltimer at the end of each step (optional)
  unsigned long long* step_rec;    // paths expanded in each step (optional)
  unsigned int step_ts_cap;
  unsigned int max_steps;          // stop after this many steps in this launch (0 = no limit)
  unsigned long long reserve;      // extra child capacity reserved for admissions (records)
  unsigned int spin_limit;
  unsigned int smem_graph;         // 1: graph data staged in shared memory
  unsigned int adj_bytes;          // bytes staged for adjacency (bitset) / rows+cols (CSR)
  unsigned int rtab_bytes;
  unsigned int seed_entries;       // CSR seeding: number of directed entries (2m)
  unsigned int* cyc_vert;          // cycle list (CSR path only): vertices, original ids
  unsigned long long* cyc_start;   // cycle i starts at cyc_vert[cyc_start[i]]
  unsigned int* cyc_len;           // and has cyc_len[i] vertices
  unsigned long long cyc_cap_c, cyc_cap_v;
  unsigned int fresh;              // 1: build frame 0 from the seed counters at kernel start
  unsigned int row_bytes;          // CSR staging: bytes of the row offsets (16-byte padded)
  unsigned long long seed_stride;  // frame 0 records per plane
  unsigned long long seed_bytes;   // frame 0 region bytes
  unsigned int cluster;            // 1: one thread-block cluster, hardware cluster barrier
  unsigned int nsig_bytes;         // CSR staging: bytes of the neighbour signatures
  const unsigned long long* nsig;  // CSR: neighbour signature of each vertex, 2 words [n]
  unsigned long long handover;     // cluster phase: stop before expanding more paths than this
  unsigned int pf;                 // bitset / batch: paths per thread per round (1..P of the kind)
  unsigned int fuse_ok;            // one graph, bitset, persistent grid: two-level steps allowed
  unsigned int cyc_stream;         // CSR cycle list drained between launches: a step takes no
                                   // more paths than the list's room allows, none when it is full
  unsigned int part, nparts;       // seeding keeps only the initial triplets (and triangles) of
                                   // this part of nparts (1 = all); see triplet_part
  unsigned int offload_min;        // host frontier on: stop (want_offload) instead of expanding a
                                   // level in chunks of fewer paths than this while frames lie
                                   // below it (0 = off)
};

// Triplet sharding: the part of the initial triplet or triangle <x, u, y> (l(u) < l(x) <
// l(y)) is mix((u n + x) n + y) mod nparts over the ORIGINAL vertex ids, so that the split
// does not depend on the labelling's tie rule or on the order in which threads find the
// triplets.  Every triplet roots its own subtree (Section 4.3), so the parts' results add
// up to the whole.
__host__ __device__ __forceinline__ unsigned int triplet_part(unsigned int x, unsigned int u, unsigned int y,
                                                              unsigned int n, unsigned int nparts) {
  const unsigned long long key = ((unsigned long long)u * n + x) * n + y;
  return (unsigned int)(mix64(key) % nparts);
}

#ifdef __CUDACC__
// Streamed CSR lists: a bound on the cycles that the child <v1 .. vt, v> closes when it is
// expanded, |Adj(v) & Adj(v1) \ {vt}| (each closing vertex neighbours both ends).  Sorted
// rows; disjoint neighbour signatures settle most pairs without reading a row.
__device__ __forceinline__ unsigned int closing_bound(const unsigned int* nrow, const unsigned short* ncol,
                                                      const unsigned long long* nsig, unsigned int v,
                                                      unsigned int v1, unsigned int vt) {
  if (((nsig[2 * v] & nsig[2 * v1]) | (nsig[2 * v + 1] & nsig[2 * v1 + 1])) == 0) return 0;
  unsigned int a = nrow[v], ae = nrow[v + 1], b = nrow[v1], be = nrow[v1 + 1], k = 0;
  while (a < ae && b < be) {
    const unsigned int x = ncol[a], y = ncol[b];
    if (x == y) {
      k += x != vt;
      ++a;
      ++b;
    } else if (x < y) {
      ++a;
    } else {
      ++b;
    }
  }
  return k;
}

// Cycle list entry in canonical order (original ids): smallest id first, then towards
// its smaller cycle neighbour.  vtx(j) returns the relabelled id of cycle position j.
template <typename F>
__device__ __forceinline__ void emit_cycle(const EngineParams& p, unsigned int k, F vtx) {
  unsigned int i0 = 0, best = p.perm[vtx(0)];
  for (unsigned int i = 1; i < k; ++i) {
    const unsigned int o = p.perm[vtx(i)];
    if (o < best) best = o, i0 = i;
  }
  const unsigned int nx = p.perm[vtx((i0 + 1) % k)], pv = p.perm[vtx((i0 + k - 1) % k)];
  const bool fwd = nx < pv;
  const unsigned long long ci = atomicAdd(&p.ctl->cyc_count, 1ull);
  const unsigned long long vb = atomicAdd(&p.ctl->cyc_verts, (unsigned long long)k);
  if (ci < p.cyc_cap_c && vb + k <= p.cyc_cap_v) {
    for (unsigned int j = 0; j < k; ++j) {
      const unsigned int idx = fwd ? (i0 + j) % k : (i0 + k - j) % k;
      p.cyc_vert[vb + j] = p.perm[vtx(idx)];
    }
    p.cyc_start[ci] = vb;
    p.cyc_len[ci] = k;
  }
}
#endif

// ------------------------------------------------------------------ small device helpers
#ifdef __CUDACC__

__device__ __forceinline__ unsigned long long ldcg64(const unsigned long long* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned int ldcg32(const unsigned int* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned short ldcg16(const unsigned short* p) { return __ldcg(p); }
__device__ __forceinline__ unsigned int ldcg8(const unsigned char* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_err(Control* ctl, int code, int info) {
  if (atomicCAS(&ctl->err, 0, code) == 0) ctl->err_info = info;
}

// Grid-wide barrier for a cooperative (co-resident) launch, with a bounded wait.
// Returns false if this block gave up waiting or any block has reported an error;
// every block then leaves its step loop, so the kernel always terminates.
__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Arrival is two-level: blocks arrive on their group's counter (kBarGroupSize blocks per
// group) and the last block of each group arrives on the grid counter, so no counter sees
// more than max(kBarGroupSize, groups) serialised atomics.  Release/acquire atomics carry
// the step's writes from every block to every block.
// `gen` is the barrier generation as last seen by this block's thread 0 (read once at
// kernel start, then advanced here), which saves a round trip per barrier.
__device__ __forceinline__ bool grid_barrier(Control* ctl, unsigned int nblocks, unsigned int spin_limit,
                                             unsigned int& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    // The arrival is an acq_rel atomic and the release a st.release: they order the
    // block's writes (made visible to thread 0 by the __syncthreads above) before every
    // block's reads after the barrier, with no separate fence on the critical path.
    int ok = 1;
    const unsigned int group = blockIdx.x / kBarGroupSize;
    const unsigned int groups = (nblocks + kBarGroupSize - 1) / kBarGroupSize;
    const unsigned int gsize = min(kBarGroupSize, nblocks - group * kBarGroupSize);
    unsigned int* gc = &ctl->bar_group[group * kBarGroupPad];
    bool last = false;
    if (atom_add_acq_rel(gc, 1u) == gsize - 1) {
      *gc = 0u;  // no block of this group touches it again before the release below
      last = atom_add_acq_rel(&ctl->bar_count, 1u) == groups - 1;
    }
    if (last) {
      ctl->bar_count = 0u;
      st_release_u32(&ctl->bar_gen, gen + 1);
    } else {
      unsigned int polls = 0;
      // poll tightly for short steps, then back off so that waiting blocks do not load
      // the memory system the working blocks need (long steps take milliseconds)
      while (ld_acquire_u32(&ctl->bar_gen) == gen) {
        if ((polls & 15) == 0 && ld_relaxed_i32(&ctl->err) != 0) { ok = 0; break; }
        if (++polls > spin_limit) { set_err(ctl, kDevTimeout, 1); ok = 0; break; }
        if (polls > 16) __nanosleep(polls < 256 ? 64 : 512);
      }
    }
    // an error raised during the step is read with the step's counters after the barrier
    gen += 1;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Exclusive block-wide prefix sum of v; *total receives the block sum.
// s_warp must hold blockDim.x/32 + 1 words; callers separate consecutive calls by a
// __syncthreads (this function ends with one).
__device__ __forceinline__ unsigned int block_exclusive_scan(unsigned int v, unsigned int* total,
                                                             unsigned int* s_warp) {
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned int w = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= (unsigned)o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  unsigned int before = wid ? s_warp[wid - 1] : 0u;
  *total = s_warp[nw - 1];
  __syncthreads();
  return before + x - v;
}

// Entry i of a warp's list of set bits, the lanes' bits in lane order (`excl` = this lane's
// exclusive prefix count of its bits): its owner is the last lane whose first entry is at
// most i (a lane without bits shares its prefix with the next lane, so for i below the
// total the last such lane has entry i).  Binary search over the lanes by shuffles; every
// lane of the warp calls it.  `rank` receives i's rank among the owner's bits.
__device__ __forceinline__ unsigned int list_owner(unsigned int excl, unsigned int i, unsigned int& rank) {
  unsigned int o = 0, eo = 0;
#pragma unroll
  for (unsigned int st = 16; st >= 1; st >>= 1) {
    const unsigned int e = __shfl_sync(0xffffffffu, excl, o + st);
    if (e <= i) {
      o += st;
      eo = e;
    }
  }
  rank = i - eo;
  return o;
}

// Index of the r-th set bit of b (r < popc(b)).
__device__ __forceinline__ unsigned int nth_set_bit(unsigned long long b, unsigned int r) {
  for (; r; --r) b &= b - 1;
  return __ffsll((long long)b) - 1;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of a u64 (result valid in thread 0).  s_red holds blockDim.x/32 words.
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* s_red) {
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_u64(v);
  __syncthreads();
  if (lane == 0) s_red[wid] = v;
  __syncthreads();
  unsigned long long r = 0;
  if (wid == 0) {
    r = lane < nw ? s_red[lane] : 0ull;
    r = warp_sum_u64(r);
  }
  return r;
}

// Output slots for one tile: each thread asks for n slots; returns the thread's first
// slot.  Warp-level inclusive scan, one block-wide combine of the warp totals by warp 0,
// one global atomic per tile on *counter.  Two __syncthreads; s_warp holds blockDim/32
// words.  Safe to call again right away (each warp reads its own offset before the next
// call's first barrier).
__device__ __forceinline__ unsigned long long tile_slots(unsigned int n, unsigned long long* counter,
                                                         unsigned int* s_warp, unsigned long long* s_base) {
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const unsigned int v = lane < nw ? s_warp[lane] : 0u;
    unsigned int vin = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, vin, o);
      if (lane >= (unsigned)o) vin += y;
    }
    const unsigned int btot = __shfl_sync(0xffffffffu, vin, 31);
    if (lane < nw) s_warp[lane] = vin - v;
    if (lane == 0) *s_base = btot ? atomicAdd(counter, (unsigned long long)btot) : 0ull;
  }
  __syncthreads();
  return *s_base + s_warp[wid] + (incl - n);
}

// Output slots for one warp: each lane asks for n slots; returns the lane's first slot.
// Warp-level inclusive scan and one global atomic per warp, no block barrier, so warps of
// a block never wait for each other.
__device__ __forceinline__ unsigned long long warp_slots(unsigned int n, unsigned long long* counter) {
  const unsigned lane = threadIdx.x & 31;
  unsigned int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  const unsigned int tot = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && tot) base = atomicAdd(counter, (unsigned long long)tot);
  return __shfl_sync(0xffffffffu, base, 31) + (incl - n);
}

// Block-wide sums of three u64 values; results valid in thread 0.  s_red: 96 words.
__device__ __forceinline__ void block_sum3_u64(unsigned long long& a, unsigned long long& b,
                                               unsigned long long& c, unsigned long long* s_red) {
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum_u64(a);
  b = warp_sum_u64(b);
  c = warp_sum_u64(c);
  __syncthreads();
  if (lane == 0) {
    s_red[wid] = a;
    s_red[32 + wid] = b;
    s_red[64 + wid] = c;
  }
  __syncthreads();
  if (wid == 0) {
    a = warp_sum_u64(lane < nw ? s_red[lane] : 0ull);
    b = warp_sum_u64(lane < nw ? s_red[32 + lane] : 0ull);
    c = warp_sum_u64(lane < nw ? s_red[64 + lane] : 0ull);
  }
}

// ---- bulk (TMA engine, non-tensor) global->shared staging with an mbarrier
__device__ __forceinline__ unsigned int smem_addr(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned int bytes,
                                              unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Asynchronous per-thread copies global -> shared (cp.async, no registers held while in
// flight); a thread waits for its own earlier groups with cp_async_wait_1.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// every group but the most recent one has landed
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
// L2 prefetch of a contiguous global range by the bulk-copy engine (no registers, no
// shared memory); address and size are multiples of 16 bytes.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned int bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

#endif  // __CUDACC__

// ------------------------------------------------------------------ host-side sizes
__host__ __device__ __forceinline__ unsigned long long round_up(unsigned long long x, unsigned long long a) {
  return (x + a - 1) / a * a;
}
// Record bytes: bitset planes (8W + 12), CSR records (2 csr_rec_u16(t)).
__host__ __device__ __forceinline__ unsigned long long bitset_region_bytes(unsigned long long stride, int W) {
  return round_up(stride * (8ull * W + 12ull), 256);
}
// Batch records: B, H (u64 planes), M (u32 plane) and N (u8 plane), 21 bytes.
__host__ __device__ __forceinline__ unsigned long long multi_region_bytes(unsigned long long stride) {
  return round_up(stride * 21ull, 256);
}
__host__ __device__ __forceinline__ unsigned int csr_rec_u16(unsigned int t) { return (t + 7u) & ~7u; }
__host__ __device__ __forceinline__ unsigned long long csr_region_bytes(unsigned long long stride, unsigned t) {
  return round_up(stride * 2ull * csr_rec_u16(t), 256);
}

// Kernel launchers (defined in the .cu files).
cudaError_t launch_label_single(const unsigned int* row_ptr, const unsigned int* col, unsigned int n,
                                unsigned int nnz, int W, unsigned int* perm, unsigned long long* adj,
                                unsigned long long* rtab, unsigned int* nrow, unsigned short* ncol,
                                unsigned long long* nsig, cudaStream_t st);
cudaError_t launch_seed_single(Kind kind, const EngineParams& p, unsigned long long seed_stride,
                               cudaStream_t st);
cudaError_t launch_engine(Kind kind, const EngineParams& p, int grid, int block, size_t smem,
                          cudaStream_t st);
cudaError_t engine_occupancy(Kind kind, int block, size_t smem, int* blocks_per_sm);
int small_cluster_size(Kind kind, size_t smem);
cudaError_t launch_small_engine(Kind kind, const EngineParams& p, int cluster, size_t smem,
                                unsigned long long handover, cudaStream_t st);
size_t engine_smem_bytes(Kind kind, const EngineParams& p, int block);
cudaError_t launch_label_seed_multi(const unsigned int* row_ptr_all, const unsigned long long* row_off,
                                    const unsigned int* col_all, const unsigned long long* col_off,
                                    const unsigned int* n_arr, const unsigned int* slot_ids, unsigned int count,
                                    unsigned int slot0, unsigned int max_len, const EngineParams& p,
                                    unsigned long long frame_base, unsigned long long stride,
                                    unsigned long long* slot_counter, unsigned long long* next_counter,
                                    cudaStream_t st);
cudaError_t launch_serve_gather(const unsigned int* slots, unsigned int count, unsigned long long* hist,
                                unsigned long long* tcount, unsigned long long* hash, unsigned long long* out,
                                cudaStream_t st);

}  // namespace cc
