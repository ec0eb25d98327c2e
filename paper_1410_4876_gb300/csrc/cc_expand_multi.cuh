// Expansion of batch and serving records (many graphs of up to 64 vertices in one frontier).
// Included by cc_engine.cu inside namespace cc, after the step plan (StepPlan, KindTraits,
// the record layouts); the persistent kernel there calls these per step.
#pragma once

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
// the hot spot of the whole grid.  The rows, r-table and L' of a record's graph (1 KB per
// graph) are read through the L1 cache at (slot << 6 | v): a copy staged in the warp's
// shared memory, with a branch for records of another graph, cost more instructions than
// the L1 hits it saved.
template <int NT>
__device__ __forceinline__ void process_multi_flat(const EngineParams& p, const StepPlan& pl,
                                                   const unsigned long long* adj, const unsigned long long* rtab) {
  constexpr int P = KindTraits<Kind::Multi>::P;
  static_assert(P == 2, "the batch form takes two paths per lane and round");
  __shared__ unsigned long long s_nb[NT / 32][P * 32];  // B | Adj(vt) per staged path
  __shared__ unsigned long long s_h[NT / 32][P * 32];   // H per staged path
  __shared__ unsigned long long s_x[NT / 32][P * 32];   // B | Adj(vt) | Adj(v1), or ~0 at t + 2 = L'
  __shared__ unsigned int s_mb[NT / 32][P * 32];        // a child's M without its v_t
  __shared__ unsigned long long s_rb[NT / 32][2][P * 32];  // records of this round and the next
  __shared__ unsigned long long s_rh[NT / 32][2][P * 32];
  __shared__ unsigned int s_rm[NT / 32][2][P * 32];
  const unsigned int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned long long* snb = s_nb[wid];
  unsigned long long* sh = s_h[wid];
  unsigned long long* sx = s_x[wid];
  unsigned int* smb = s_mb[wid];  // v1 | (t + 1) << 12 | g << 18
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
  auto A = [&](unsigned int g, unsigned int v) -> unsigned long long {
    return __ldg(adj + ((g << 6) | v));
  };
  auto R = [&](unsigned int g, unsigned int v) -> unsigned long long {
    return __ldg(rtab + ((g << 6) | v));
  };

  unsigned long long m[P] = {};
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
    __syncwarp();  // the staged paths (snb, sh, sx, smb) of every lane
    for (unsigned int w0 = 0; w0 < n; w0 += 32) {
      const unsigned int i = w0 + lane;
      unsigned int k;
      const unsigned int o = list_owner(excl, i, k);
      const unsigned long long b0 = __shfl_sync(0xffffffffu, m[0], o), b1 = __shfl_sync(0xffffffffu, m[1], o);
      const unsigned int c0o = __shfl_sync(0xffffffffu, c0n, o);
      if (i < n) {
        unsigned int j = 0;
        unsigned long long b = b0;
        if (k >= c0o) {
          k -= c0o;
          j = 1;
          b = b1;
        }
        const unsigned int v = nth_set_bit(b, k), pj = j * 32u + o;
        const unsigned int mb = smb[pj], g = mb >> 18;
        const unsigned int slot = base + i;
        if (slot < ds32) {
          const unsigned long long nb = snb[pj];
          dB[slot] = nb;
          dH[slot] = sh[pj] + R(g, v);
          dM[slot] = mb | (v << 6);
          // the child's own children: Adj(v) minus its blocked set and Adj(v1)
          const unsigned int nc = __popcll(A(g, v) & ~sx[pj]);
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
        const unsigned int Lr = valid ? __ldg(p.Lg + g) : 0u;
        const unsigned long long at = A(g, vt), a1 = A(g, v1);
        const unsigned long long cand = at & ~B;
        m[j] = (tt + 1 <= Lr) ? (cand & a1) : 0ull;
        ch[j] = (store && tt + 1 < Lr) ? (cand & ~a1) : 0ull;
        const unsigned int pj = j * 32 + lane;
        snb[pj] = B | at;
        sh[pj] = H;
        sx[pj] = (tt + 2 < Lr) ? (B | at | a1) : ~0ull;
        smb[pj] = v1 | ((tt + 1) << 12) | (g << 18);
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
