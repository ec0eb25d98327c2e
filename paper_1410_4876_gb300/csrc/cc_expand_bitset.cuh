// Expansion of one graph's bitset records: the flattened and two-level forms of the persistent
// grid, and the per-lane forms of the small-level cluster phase.
// Included by cc_engine.cu inside namespace cc, after the step plan (StepPlan, KindTraits,
// the record layouts); the persistent kernel there calls these per step.
#pragma once

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
