// Degree labelling (Section 2) and initial triplets / triangles (Section 4.3, Algorithm 2).
//
// The labelling is inherently sequential (Section 4 keeps it on the host; Section 6 proposes
// degree updates by one processor per edge and a parallel minimum per step); here one warp
// runs it on the device so the whole enumeration stays on the GPU with no host round
// trip.  Each step takes the live vertex of minimum current degree (ties: smallest id),
// found by one warp reduction over a two-level tree of minima (32-vertex groups, 32-group
// supergroups), while the lanes lower its neighbours' degrees in parallel.  Vertices are then renumbered by label (new id = label - 1),
// so "l(x) < l(y)" becomes "x < y" and every label test is an integer or bit-mask test.
//
// Seeding replaces the |V| * Delta^2 flat thread grid of Algorithm 2 (most of whose
// threads fall outside the neighbour range) by one thread per (u, x) pair of a
// relabelled adjacency row; the pairs y > x come out of one mask operation.
#include <mutex>

#include "cc_internal.cuh"

namespace cc {

// ------------------------------------------------------------------ labelling, one graph

// Dynamic shared memory: key[n] (u32), gmin[G] (u32), sgmin[32] (u32), G = ceil(n / 32).
// key(v) = current_degree << 16 | v for a live vertex, 0xFFFFFFFF once removed.  gmin[g]
// is the smallest key of the 32 vertices of group g, sgmin[s] the smallest of the 32 group
// minima of supergroup s (n <= 32768 gives at most 32 supergroups, one per lane).
//
// Each step of the labelling (Section 2: remove a vertex of minimum current degree, ties
// by smallest id) is one warp reduction over sgmin (over gmin directly when there are at
// most 64 groups).  Removing u lowers its neighbours'
// keys, and only keys of u's own group and supergroup can rise (u's key becomes dead), so
// a step recomputes gmin of u's group (one load per lane: the group's keys, with the
// neighbours' new keys folded in) and sgmin of u's supergroup (one load per lane), and
// lowers every other affected minimum by atomicMin.  The row of u, its neighbours' keys
// and the group's keys are loaded side by side, so a step is a short chain of dependent
// shared-memory accesses and two reductions.
__global__ void __launch_bounds__(1024) label_single_kernel(const unsigned int* __restrict__ row_ptr,
                                                            const unsigned int* __restrict__ col, unsigned int n,
                                                            int W, unsigned int* perm, unsigned int* newid,
                                                            unsigned long long* adj, unsigned long long* rtab,
                                                            unsigned int* nrow, unsigned short* ncol,
                                                            unsigned long long* nsig, int stage_csr) {
  extern __shared__ unsigned int sm_label[];
  unsigned int* key = sm_label;
  const unsigned int G = (n + 31) / 32;
  unsigned int* gmin = sm_label + n;
  unsigned int* sgmin = gmin + G;
  const unsigned int tid = threadIdx.x, lane = tid & 31;
  const unsigned int kDead = 0xFFFFFFFFu;
  if (stage_csr) {
    // the sequential loop below reads a row per step: keep the CSR in shared memory
    unsigned int* rp_s = sgmin + 32;
    unsigned int* col_s = rp_s + n + 1;
    const unsigned int nnz = row_ptr[n];
    for (unsigned int i = tid; i <= n; i += blockDim.x) rp_s[i] = row_ptr[i];
    for (unsigned int i = tid; i < nnz; i += blockDim.x) col_s[i] = col[i];
    __syncthreads();
    row_ptr = rp_s;
    col = col_s;
  }
  for (unsigned int v = tid; v < n; v += blockDim.x) key[v] = ((row_ptr[v + 1] - row_ptr[v]) << 16) | v;
  __syncthreads();
  for (unsigned int g = tid; g < G; g += blockDim.x) {
    unsigned int m = kDead;
    for (unsigned int j = 0; j < 32; ++j) {
      const unsigned int v = g * 32 + j;
      if (v < n) m = min(m, key[v]);
    }
    gmin[g] = m;
  }
  __syncthreads();
  if (tid < 32) {
    {
      unsigned int m = kDead;
      for (unsigned int g = lane * 32; g < G && g < lane * 32 + 32; ++g) m = min(m, gmin[g]);
      sgmin[lane] = m;  // (lanes past the last supergroup hold dead)
    }
    __syncwarp();
    // up to 64 groups (n <= 2048): the step's minimum straight from the group minima, two
    // per lane, and no supergroup level to keep
    const bool flat = G <= 64;
    for (unsigned int i = 0; i < n; ++i) {
      const unsigned int m = flat ? __reduce_min_sync(0xffffffffu, min(lane < G ? gmin[lane] : kDead,
                                                                       lane + 32 < G ? gmin[lane + 32] : kDead))
                                  : __reduce_min_sync(0xffffffffu, sgmin[lane]);
      const unsigned int u = m & 0xFFFFu, gu = u >> 5, su = gu >> 5;
      // u's group without u, and u's row (loaded side by side)
      const unsigned int v = gu * 32 + lane;
      unsigned int kg = (v < n && v != u) ? key[v] : kDead;
      const unsigned int rb = row_ptr[u], re = row_ptr[u + 1];
      for (unsigned int e = rb + lane; e < re; e += 32) {
        const unsigned int w = col[e];
        unsigned int kw = key[w];
        if (kw != kDead) {
          kw -= 1u << 16;
          key[w] = kw;
          const unsigned int gw = w >> 5;
          if (gw == gu) {
            kg = min(kg, kw);
          } else {
            atomicMin(&gmin[gw], kw);
            if (!flat && (gw >> 5) != su) atomicMin(&sgmin[gw >> 5], kw);
          }
        }
      }
      kg = __reduce_min_sync(0xffffffffu, kg);
      if (lane == 0) {
        gmin[gu] = kg;
        key[u] = kDead;
        perm[i] = u;
        newid[u] = i;
      }
      __syncwarp();
      if (!flat) {
        // u's supergroup: its groups' minima after this step's updates
        const unsigned int g2 = su * 32 + lane;
        const unsigned int ks = __reduce_min_sync(0xffffffffu, g2 < G ? gmin[g2] : kDead);
        if (lane == 0) sgmin[su] = ks;
        __syncwarp();
      }
    }
  }
  __syncthreads();

  for (unsigned int v = tid; v < n; v += blockDim.x) rtab[newid[v]] = vertex_r(v);
  if ((n & 1) && tid == 0) rtab[n] = 0;  // 16-byte padding of the staged copy

  if (W > 0) {
    // bitset rows in new ids; row r lists the new ids of perm[r]'s neighbours
    const unsigned int npad = (n + 1) & ~1u;
    for (unsigned int r = tid; r < npad; r += blockDim.x) {
      unsigned long long w[4] = {0, 0, 0, 0};
      if (r < n) {
        const unsigned int v = perm[r];
        for (unsigned int e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
          const unsigned int x = newid[col[e]];
          w[x >> 6] |= 1ull << (x & 63);
        }
      }
      for (int k = 0; k < W; ++k) adj[(unsigned long long)r * W + k] = w[k];
    }
    return;
  }

  // CSR in new ids: row offsets by a block scan of the degrees in label order ...
  __shared__ unsigned int s_warp[33];
  const unsigned int per = (n + blockDim.x - 1) / blockDim.x;
  const unsigned int r0 = min(n, tid * per), r1 = min(n, r0 + per);
  unsigned int local = 0;
  for (unsigned int r = r0; r < r1; ++r) local += row_ptr[perm[r] + 1] - row_ptr[perm[r]];
  unsigned int total;
  unsigned int run = block_exclusive_scan(local, &total, s_warp);
  for (unsigned int r = r0; r < r1; ++r) {
    nrow[r] = run;
    run += row_ptr[perm[r] + 1] - row_ptr[perm[r]];
  }
  if (tid == 0) nrow[n] = total;
  __syncthreads();
  // ... then each row sorted by rank (one warp per row; ids within a row are distinct),
  // and the row's neighbour signature (OR of sig_bit over the row) next to it
  const unsigned int warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (unsigned int r = warp; r < n; r += nwarps) {
    const unsigned int v = perm[r], b = row_ptr[v], d = row_ptr[v + 1] - b, out = nrow[r];
    unsigned int sg[4] = {0, 0, 0, 0};
    for (unsigned int a = lane; a < d; a += 32) {
      const unsigned int x = newid[col[b + a]];
      unsigned int rank = 0;
      for (unsigned int c = 0; c < d; ++c) rank += newid[col[b + c]] < x;
      ncol[out + rank] = (unsigned short)x;
      const unsigned int sb = sig_bit(x);
      sg[sb >> 5] |= 1u << (sb & 31u);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) sg[k] = __reduce_or_sync(0xffffffffu, sg[k]);
    if (lane == 0) {
      nsig[2ull * r] = (unsigned long long)sg[1] << 32 | sg[0];
      nsig[2ull * r + 1] = (unsigned long long)sg[3] << 32 | sg[2];
    }
  }
}

// The same labelling for n <= 64 with one-word rows: one warp, every vertex's adjacency
// row and current degree in registers (lane l owns vertices l and l + 32), one warp
// reduction per step and no shared or global memory inside the sequential loop.
__global__ void __launch_bounds__(32) label_small_kernel(const unsigned int* __restrict__ row_ptr,
                                                         const unsigned int* __restrict__ col, unsigned int n,
                                                         unsigned int* perm, unsigned int* newid,
                                                         unsigned long long* adj, unsigned long long* rtab) {
  __shared__ unsigned char s_nid[64];
  const unsigned int lane = threadIdx.x;
  unsigned long long ao[2] = {0, 0};
  unsigned int deg[2] = {0, 0};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const unsigned int v = lane + 32u * k;
    if (v < n) {
      for (unsigned int e = row_ptr[v]; e < row_ptr[v + 1]; ++e) ao[k] |= 1ull << col[e];
      deg[k] = row_ptr[v + 1] - row_ptr[v];
    }
  }
  unsigned long long alive = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
  for (unsigned int i = 0; i < n; ++i) {
    unsigned int key = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const unsigned int v = lane + 32u * k;
      if (v < n && ((alive >> v) & 1ull)) key = min(key, (deg[k] << 8) | v);
    }
    key = __reduce_min_sync(0xffffffffu, key);
    const unsigned int u = key & 0xFFu;
    if (lane == 0) {
      s_nid[u] = (unsigned char)i;
      perm[i] = u;
      newid[u] = i;
    }
    alive &= ~(1ull << u);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const unsigned int v = lane + 32u * k;
      if (v < n && ((alive >> v) & 1ull) && ((ao[k] >> u) & 1ull)) deg[k] -= 1;
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const unsigned int v = lane + 32u * k;
    if (v < n) {
      unsigned long long row = 0, b = ao[k];
      while (b) {
        const unsigned int w = __ffsll((long long)b) - 1;
        b &= b - 1;
        row |= 1ull << s_nid[w];
      }
      adj[s_nid[v]] = row;
      rtab[s_nid[v]] = vertex_r(v);
    }
  }
  // 16-byte padding of the staged copies
  if (lane == 0 && (n & 1)) {
    adj[n] = 0;
    rtab[n] = 0;
  }
}

cudaError_t launch_label_single(const unsigned int* row_ptr, const unsigned int* col, unsigned int n,
                                unsigned int nnz, int W, unsigned int* perm, unsigned long long* adj,
                                unsigned long long* rtab, unsigned int* nrow, unsigned short* ncol,
                                unsigned long long* nsig, cudaStream_t st) {
  if (W == 1 && n <= 64) {
    label_small_kernel<<<1, 32, 0, st>>>(row_ptr, col, n, perm, perm + n, adj, rtab);
    return cudaGetLastError();
  }
  // perm holds 2n words: perm[0..n) new->original, perm[n..2n) original->new
  size_t smem = sizeof(unsigned int) * (n + (n + 31) / 32 + 32);
  const size_t csr_words = (size_t)n + 1 + nnz;
  const int stage = (smem + 4 * csr_words) <= 96 * 1024 ? 1 : 0;
  if (stage) smem += 4 * csr_words;
  // the limit is only raised (a replayed CUDA graph of a larger graph keeps its node's size)
  static std::mutex mu;
  static size_t allowed = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (smem > allowed) {
      cudaError_t e = cudaFuncSetAttribute(label_single_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      allowed = smem;
    }
  }
  label_single_kernel<<<1, 1024, smem, st>>>(row_ptr, col, n, W, perm, perm + n, adj, rtab, nrow, ncol, nsig, stage);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ helpers on W-word masks

template <int W>
__device__ __forceinline__ void mask_low(unsigned long long (&m)[W], unsigned int u) {
  // bits 0..u set (every vertex whose label is <= l(u))
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const unsigned int lo = 64u * k;
    if (u >= lo + 63) m[k] = ~0ull;
    else if (u < lo) m[k] = 0ull;
    else m[k] = (2ull << (u - lo)) - 1ull;
  }
}

// ------------------------------------------------------------------ seeding, one graph, bitset

// Frame 0 planes at arena offset 0 with the given stride.  One thread per (u, x).
template <int W>
__global__ void __launch_bounds__(256) seed_bitset_kernel(EngineParams p, unsigned long long stride) {
  const unsigned int n = p.n, L = p.L;
  const unsigned long long id = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned int lane = threadIdx.x & 31;
  const unsigned long long* adj = p.adj;
  const unsigned long long* rtab = p.rtab;
  unsigned int u = 0, x = 0;
  bool active = false;
  if (id < (unsigned long long)n * n) {
    u = (unsigned int)(id / n);
    x = (unsigned int)(id % n);
    active = x > u && ((adj[(unsigned long long)u * W + (x >> 6)] >> (x & 63)) & 1ull);
  }
  unsigned long long au[W], ax[W], ys[W], paths[W];
  unsigned long long ntri = 0, hacc = 0;
  unsigned int npath = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    au[k] = active ? adj[(unsigned long long)u * W + k] : 0ull;
    ax[k] = active ? adj[(unsigned long long)x * W + k] : 0ull;
  }
  unsigned long long lowx[W];
  mask_low<W>(lowx, x);
#pragma unroll
  for (int k = 0; k < W; ++k) {
    ys[k] = au[k] & ~lowx[k];           // y in Adj(u), y > x  (so l(u) < l(x) < l(y))
    if (p.nparts > 1 && ys[k]) {         // triplet sharding: keep this part's triplets only
      const unsigned int ox = p.perm[x], ou = p.perm[u];
      unsigned long long b = ys[k], keep = 0ull;
      while (b) {
        const unsigned int y = 64u * k + __ffsll((long long)b) - 1;
        if (triplet_part(ox, ou, p.perm[y], n, p.nparts) == p.part) keep |= b & (0ull - b);
        b &= b - 1;
      }
      ys[k] = keep;
    }
    const unsigned long long tri = ys[k] & ax[k];    // (x, y) in E: triangle
    paths[k] = (L > 3) ? (ys[k] & ~ax[k]) : 0ull;    // otherwise an initial chordless path
    ntri += __popcll(tri);
    npath += __popcll(paths[k]);
    unsigned long long b = tri;
    while (b) {
      const unsigned int y = 64u * k + __ffsll((long long)b) - 1;
      b &= b - 1;
      hacc += mix64(rtab[x] + rtab[u] + rtab[y] + 3ull * kGamma);
    }
  }
  if (L < 3) ntri = 0, hacc = 0;
  // warp-aggregated slot allocation
  unsigned int incl = npath;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  const unsigned int wtot = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && wtot) base = atomicAdd(&p.ctl->seed_count, (unsigned long long)wtot);
  base = __shfl_sync(0xffffffffu, base, 31) + (incl - npath);
  unsigned long long nx = 0;
  if (npath) {
    unsigned long long B[W];
    mask_low<W>(B, u);
#pragma unroll
    for (int k = 0; k < W; ++k) B[k] |= au[k];      // interior {u}: Adj(u), plus labels <= l(u)
    const unsigned long long H0 = rtab[x] + rtab[u];
    unsigned long long* dB = (unsigned long long*)p.arena;
    unsigned long long* dH = dB + (unsigned long long)W * stride;
    unsigned int* dM = (unsigned int*)(dH + stride);
    unsigned long long slot = base;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      unsigned long long b = paths[k];
      while (b) {
        const unsigned int y = 64u * k + __ffsll((long long)b) - 1;
        b &= b - 1;
        if (slot >= stride) { set_err(p.ctl, kDevSeedCap, 0); break; }
#pragma unroll
        for (int q = 0; q < W; ++q) dB[(unsigned long long)q * stride + slot] = B[q];
        dH[slot] = H0 + rtab[y];
        dM[slot] = x | (y << 16);
        if (L > 4) {
#pragma unroll
          for (int q = 0; q < W; ++q) nx += __popcll(adj[(unsigned long long)y * W + q] & ~B[q] & ~ax[q]);
        }
        ++slot;
      }
    }
  }
  // reductions
  ntri = warp_sum_u64(ntri);
  hacc = warp_sum_u64(hacc);
  nx = warp_sum_u64(nx);
  unsigned long long np = warp_sum_u64(npath);
  if (lane == 0) {
    if (ntri) atomicAdd(&p.hist[3], ntri);
    if (hacc) atomicAdd(p.hash, hacc);
    if (nx) atomicAdd(&p.ctl->seed_next, nx);
    if (np) atomicAdd(&p.tcount[3], np);
  }
}

// ------------------------------------------------------------------ seeding, one graph, CSR

__device__ __forceinline__ bool csr_adjacent(const unsigned int* nrow, const unsigned short* ncol, unsigned int a,
                                             unsigned int b) {
  unsigned int lo = nrow[a], hi = nrow[a + 1];
  while (lo < hi) {
    const unsigned int mid = (lo + hi) >> 1;
    const unsigned int c = ncol[mid];
    if (c == b) return true;
    if (c < b) lo = mid + 1; else hi = mid;
  }
  return false;
}

// One thread per directed CSR entry (u, x) with x > u.  Frame 0: one record per triplet.
__global__ void __launch_bounds__(256) seed_csr_kernel(EngineParams p, unsigned long long stride) {
  const unsigned int n = p.n, L = p.L;
  const unsigned int m2 = p.nrow[n];
  const unsigned int e = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned int lane = threadIdx.x & 31;
  unsigned int u = 0, x = 0, rend = 0;
  bool active = false;
  if (e < m2) {
    unsigned int lo = 0, hi = n;  // owner row: largest u with nrow[u] <= e
    while (hi - lo > 1) {
      const unsigned int mid = (lo + hi) >> 1;
      if (p.nrow[mid] <= e) lo = mid; else hi = mid;
    }
    u = lo;
    x = p.ncol[e];
    rend = p.nrow[u + 1];
    active = x > u;
  }
  unsigned long long ntri = 0, hacc = 0;
  unsigned int npath = 0;
  const bool split = p.nparts > 1;
  const unsigned int ox = split && active ? p.perm[x] : 0u, ou = split && active ? p.perm[u] : 0u;
  if (active && L >= 3) {
    for (unsigned int f = e + 1; f < rend; ++f) {  // rows are sorted: y > x
      const unsigned int y = p.ncol[f];
      if (split && triplet_part(ox, ou, p.perm[y], n, p.nparts) != p.part) continue;
      if (csr_adjacent(p.nrow, p.ncol, x, y)) {
        ++ntri;
        hacc += mix64(p.rtab[x] + p.rtab[u] + p.rtab[y] + 3ull * kGamma);
        if (p.cyc_vert) {
          const unsigned int c[3] = {x, u, y};
          emit_cycle(p, 3, [&](unsigned int j) { return c[j]; });
        }
      } else if (L > 3) {
        ++npath;
      }
    }
  }
  unsigned int incl = npath;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  const unsigned int wtot = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && wtot) base = atomicAdd(&p.ctl->seed_count, (unsigned long long)wtot);
  base = __shfl_sync(0xffffffffu, base, 31) + (incl - npath);
  unsigned long long nb = 0;
  if (npath) {
    uint4* R0 = reinterpret_cast<uint4*>(p.arena);  // one 8-id record per triplet
    unsigned long long slot = base;
    for (unsigned int f = e + 1; f < rend; ++f) {
      const unsigned int y = p.ncol[f];
      if (split && triplet_part(ox, ou, p.perm[y], n, p.nparts) != p.part) continue;
      if (csr_adjacent(p.nrow, p.ncol, x, y)) continue;
      if (slot >= stride) { set_err(p.ctl, kDevSeedCap, 0); break; }
      R0[slot] = make_uint4(x | (u << 16), y | 0xFFFF0000u, 0xFFFFFFFFu, 0xFFFFFFFFu);
      if (L > 4) nb += p.nrow[y + 1] - p.nrow[y] - 1;  // bound on this path's children
      ++slot;
    }
  }
  ntri = warp_sum_u64(ntri);
  hacc = warp_sum_u64(hacc);
  nb = warp_sum_u64(nb);
  unsigned long long np = warp_sum_u64(npath);
  if (lane == 0) {
    if (ntri) atomicAdd(&p.hist[3], ntri);
    if (hacc) atomicAdd(p.hash, hacc);
    if (np) atomicAdd(&p.tcount[3], np);
    if (nb) atomicAdd(&p.ctl->seed_next, nb);
  }
}

cudaError_t launch_seed_single(Kind kind, const EngineParams& p, unsigned long long seed_stride, cudaStream_t st) {
  if (is_csr(kind)) {
    // one thread per CSR entry; row_ptr[n] is known on the host as 2m (passed via adj_bytes)
    const unsigned int m2 = p.seed_entries;
    const unsigned int blocks = (m2 + 255) / 256;
    if (blocks) seed_csr_kernel<<<blocks, 256, 0, st>>>(p, seed_stride);
    return cudaGetLastError();
  }
  const unsigned long long threads = (unsigned long long)p.n * p.n;
  const unsigned int blocks = (unsigned int)((threads + 255) / 256);
  if (!blocks) return cudaSuccess;
  switch (kind) {
    case Kind::Bitset1: seed_bitset_kernel<1><<<blocks, 256, 0, st>>>(p, seed_stride); break;
    case Kind::Bitset2: seed_bitset_kernel<2><<<blocks, 256, 0, st>>>(p, seed_stride); break;
    case Kind::Bitset4: seed_bitset_kernel<4><<<blocks, 256, 0, st>>>(p, seed_stride); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ batch: label + seed

// One warp per graph (n <= 64).  Lane l owns original vertices l and l + 32.  The
// relabelled rows and r-table are written to the slot's region of p.adj / p.rtab and the
// initial triplets are appended to the frame described by (base, stride, counters).
__global__ void __launch_bounds__(128) label_seed_multi_kernel(
    const unsigned int* __restrict__ row_ptr_all, const unsigned long long* __restrict__ row_off,
    const unsigned int* __restrict__ col_all, const unsigned long long* __restrict__ col_off,
    const unsigned int* __restrict__ n_arr, const unsigned int* __restrict__ slot_ids, unsigned int count,
    unsigned int slot0, unsigned int max_len, EngineParams p, unsigned long long frame_base,
    unsigned long long stride, unsigned long long* slot_counter, unsigned long long* next_counter) {
  __shared__ unsigned long long s_row[4][64];
  __shared__ unsigned long long s_r[4][64];
  __shared__ unsigned char s_nid[4][64];
  const unsigned int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const unsigned int gi = blockIdx.x * 4 + wl;
  if (gi >= count) return;
  const unsigned int slot = slot_ids ? slot_ids[gi] : slot0 + gi;
  const unsigned int n = n_arr[gi];
  const unsigned int* rp = row_ptr_all + row_off[gi];
  const unsigned int* cl = col_all + col_off[gi];
  unsigned long long ao[2] = {0, 0};
  unsigned int deg[2] = {0, 0};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const unsigned int v = lane + 32u * k;
    if (v < n) {
      for (unsigned int e = rp[v]; e < rp[v + 1]; ++e) ao[k] |= 1ull << cl[e];
      deg[k] = rp[v + 1] - rp[v];
    }
  }
  // degree labelling (Section 2), ties by smallest id
  unsigned long long alive = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
  for (unsigned int i = 0; i < n; ++i) {
    unsigned int key = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const unsigned int v = lane + 32u * k;
      if (v < n && ((alive >> v) & 1ull)) key = min(key, (deg[k] << 8) | v);
    }
    key = __reduce_min_sync(0xffffffffu, key);
    const unsigned int u = key & 0xFFu;
    if (lane == 0) s_nid[wl][u] = (unsigned char)i;
    alive &= ~(1ull << u);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const unsigned int v = lane + 32u * k;
      if (v < n && ((alive >> v) & 1ull) && ((ao[k] >> u) & 1ull)) deg[k] -= 1;
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const unsigned int v = lane + 32u * k;
    if (v < n) {
      unsigned long long row = 0, b = ao[k];
      while (b) {
        const unsigned int w = __ffsll((long long)b) - 1;
        b &= b - 1;
        row |= 1ull << s_nid[wl][w];
      }
      const unsigned int r = s_nid[wl][v];
      s_row[wl][r] = row;
      s_r[wl][r] = vertex_r(v);
      const_cast<unsigned long long*>(p.adj)[(unsigned long long)slot * 64 + r] = row;
      const_cast<unsigned long long*>(p.rtab)[(unsigned long long)slot * 64 + r] = vertex_r(v);
    }
  }
  __syncwarp();
  const unsigned int L = (max_len == 0 || max_len > n) ? n : max_len;
  if (lane == 0) p.Lg[slot] = (unsigned char)L;
  // initial triplets and triangles
  unsigned long long ntri = 0, hacc = 0;
  unsigned int npath = 0;
  for (unsigned int u = lane; u < n; u += 32) {
    const unsigned long long au = s_row[wl][u];
    unsigned long long xs = au & ~((2ull << u) - 1ull);
    while (xs) {
      const unsigned int x = __ffsll((long long)xs) - 1;
      xs &= xs - 1;
      const unsigned long long ys = au & ~((2ull << x) - 1ull);
      const unsigned long long tri = ys & s_row[wl][x];
      ntri += __popcll(tri);
      unsigned long long b = tri;
      while (b) {
        const unsigned int y = __ffsll((long long)b) - 1;
        b &= b - 1;
        hacc += mix64(s_r[wl][x] + s_r[wl][u] + s_r[wl][y] + 3ull * kGamma);
      }
      if (L > 3) npath += __popcll(ys & ~s_row[wl][x]);
    }
  }
  if (L < 3) ntri = 0, hacc = 0;
  unsigned int incl = npath;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  const unsigned int wtot = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && wtot) base = atomicAdd(slot_counter, (unsigned long long)wtot);
  base = __shfl_sync(0xffffffffu, base, 31) + (incl - npath);
  unsigned long long nx = 0;
  if (npath) {
    unsigned long long* dB = (unsigned long long*)(p.arena + frame_base);
    unsigned long long* dH = dB + stride;
    unsigned int* dM = (unsigned int*)(dH + stride);
    unsigned char* dN = (unsigned char*)(dM + stride);
    unsigned long long slotpos = base;
    for (unsigned int u = lane; u < n; u += 32) {
      const unsigned long long au = s_row[wl][u];
      const unsigned long long B = au | ((2ull << u) - 1ull);
      unsigned long long xs = au & ~((2ull << u) - 1ull);
      while (xs) {
        const unsigned int x = __ffsll((long long)xs) - 1;
        xs &= xs - 1;
        unsigned long long ps = au & ~((2ull << x) - 1ull) & ~s_row[wl][x];
        while (ps) {
          const unsigned int y = __ffsll((long long)ps) - 1;
          ps &= ps - 1;
          if (slotpos >= stride) { set_err(p.ctl, kDevSeedCap, 1); ps = 0; xs = 0; break; }
          dB[slotpos] = B;
          dH[slotpos] = s_r[wl][x] + s_r[wl][u] + s_r[wl][y];
          dM[slotpos] = x | (y << 6) | (3u << 12) | (slot << 18);
          const unsigned int nc = (L > 4) ? __popcll(s_row[wl][y] & ~B & ~s_row[wl][x]) : 0u;
          dN[slotpos] = (unsigned char)nc;  // the triplet's exact child count
          nx += nc;
          ++slotpos;
        }
      }
    }
  }
  ntri = warp_sum_u64(ntri);
  hacc = warp_sum_u64(hacc);
  nx = warp_sum_u64(nx);
  const unsigned long long np = warp_sum_u64(npath);
  if (lane == 0) {
    const unsigned long long h = (unsigned long long)slot * kMultiHistStride;
    if (ntri) atomicAdd(&p.hist[h + 3], ntri);
    if (hacc) atomicAdd(&p.hash[slot], hacc);
    if (np) atomicAdd(&p.tcount[h + 3], np);
    if (nx) atomicAdd(next_counter, nx);
    if (p.live) atomicAdd((unsigned long long*)&p.live[slot], np);
  }
}

cudaError_t launch_label_seed_multi(const unsigned int* row_ptr_all, const unsigned long long* row_off,
                                    const unsigned int* col_all, const unsigned long long* col_off,
                                    const unsigned int* n_arr, const unsigned int* slot_ids, unsigned int count,
                                    unsigned int slot0, unsigned int max_len, const EngineParams& p,
                                    unsigned long long frame_base, unsigned long long stride,
                                    unsigned long long* slot_counter, unsigned long long* next_counter,
                                    cudaStream_t st) {
  if (!count) return cudaSuccess;
  label_seed_multi_kernel<<<(count + 3) / 4, 128, 0, st>>>(row_ptr_all, row_off, col_all, col_off, n_arr, slot_ids,
                                                           count, slot0, max_len, p, frame_base, stride,
                                                           slot_counter, next_counter);
  return cudaGetLastError();
}

}  // namespace cc
