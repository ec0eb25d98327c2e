// Expansion of CSR records (one graph of up to 32768 vertices; paths as u16 id rows).
// Included by cc_engine.cu inside namespace cc, after the step plan (StepPlan, KindTraits,
// the record layouts); the persistent kernel there calls these per step.
#pragma once

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
