// Serving: continuous batching of enumeration requests on one persistent frontier.
//
// Every in-flight request owns a slot (relabelled adjacency, hash table, length bound,
// histogram, hash, level counts and a count of its paths still in flight).  All paths of
// all slots share the batch engine's frontier; each record carries its slot and length,
// so paths of requests admitted at different times are expanded side by side in the same
// steps.  Between rounds of steps the host
//   - reads the in-flight counts (one copy) and gathers the results of slots at zero,
//   - admits queued requests into free slots, subject to a budget of predicted frontier
//     bytes, and appends their initial triplets to the top frame of the live frontier
//     (every frame the engine creates keeps reserve_paths free records for this),
//   - resumes the engine for steps_per_round steps.
#include <chrono>
#include <cmath>
#include <deque>
#include <thread>

#include "cc_host.hpp"

namespace {

constexpr int kHistW = kMultiHistStride;  // 65
// coefficients of the peak-path predictor (see cc_serve_predict_bytes)
constexpr double kPredC[5] = {-2.8467 + 0.9387, 0.215332, 1.239567, -0.192495, -0.045087};
constexpr int kOutW = 2 * kHistW + 1;     // hist | tcount | hash per gathered slot

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id;
  uint32_t n;
  std::vector<uint32_t> rows, cols;
  uint64_t pred_bytes;
  uint64_t seed_bound;  // (max_degree - 1) * m / 2: bound on its initial triplets
  uint32_t maxch;       // max_degree - 1 (at least 1): children per path at most
  Clock::time_point t_submit;
};

struct SlotState {
  bool busy = false;
  uint64_t id = 0;
  uint64_t pred_bytes = 0;
  uint32_t maxch = 1, L = 3;  // the request's children-per-path bound and L
  Clock::time_point t_submit, t_admit;
};

__global__ void serve_gather_kernel(const unsigned int* slots, unsigned int count, unsigned long long* hist,
                                    unsigned long long* tcount, unsigned long long* hash, unsigned long long* out) {
  const unsigned int i = blockIdx.x;
  if (i >= count) return;
  const unsigned long long s = slots[i];
  for (unsigned int k = threadIdx.x; k < kHistW; k += blockDim.x) {
    out[(unsigned long long)i * kOutW + k] = hist[s * kHistW + k];
    out[(unsigned long long)i * kOutW + kHistW + k] = tcount[s * kHistW + k];
    hist[s * kHistW + k] = 0;
    tcount[s * kHistW + k] = 0;
  }
  if (threadIdx.x == 0) {
    out[(unsigned long long)i * kOutW + 2 * kHistW] = hash[s];
    hash[s] = 0;
  }
}

}  // namespace

namespace cc {
cudaError_t launch_serve_gather(const unsigned int* slots, unsigned int count, unsigned long long* hist,
                                unsigned long long* tcount, unsigned long long* hash, unsigned long long* out,
                                cudaStream_t st) {
  if (!count) return cudaSuccess;
  serve_gather_kernel<<<count, 64, 0, st>>>(slots, count, hist, tcount, hash, out);
  return cudaGetLastError();
}
}  // namespace cc

struct cc_server {
  cc_context* ctx = nullptr;
  cc_serve_options o{};
  unsigned int slots = 0;
  // device: per-slot tables
  unsigned char* d_tab = nullptr;
  unsigned long long *d_adj = nullptr, *d_rtab = nullptr, *d_hist = nullptr, *d_hash = nullptr,
                     *d_tcount = nullptr;
  long long* d_live = nullptr;
  unsigned char* d_Lg = nullptr;
  unsigned long long* d_dummy = nullptr;
  // device + pinned host staging for uploads, status and gathers
  unsigned char* d_up = nullptr;
  unsigned char* h_up = nullptr;
  size_t up_bytes = 0;
  unsigned long long* d_out = nullptr;
  unsigned long long* h_out = nullptr;
  unsigned int* d_gslots = nullptr;
  unsigned int* h_gslots = nullptr;
  unsigned char* h_status = nullptr;  // Control | top Frame | live[slots]
  size_t status_bytes = 0;
  // host
  std::deque<Request> queue;
  std::vector<SlotState> st;
  std::vector<unsigned int> free_slots;
  std::deque<cc_completion> done;
  uint64_t next_id = 1;
  uint64_t pred_in_flight = 0;
  unsigned int in_flight = 0;
  EngineParams p{};
  int grid = 0, block = 256;
  bool launched = false;
  // requests in flight by children-per-path bound and by L': the engine's chunk planning
  // uses the largest of each (a frontier holds only paths of requests in flight)
  unsigned int n_maxch[kMultiMaxN + 1] = {};
  unsigned int n_L[kMultiMaxN + 1] = {};
};

// ------------------------------------------------------------------ prediction

// Predicted peak of stored chordless paths, from a least-squares fit of
// log(peak + 1) = c0 + c1 n + c2 (2m/n) + c3 max_degree + c4 (2m/n)^2 over 1536 measured
// graphs of the request families served here (1200 batch-mixture members: G(n, p) with n
// in [16, 64] and p in [0.08, 0.3], k x l grids with k, l in [3, 6], K_{a,b} with a, b in
// [2, 8]; 300 serving requests; every grid up to 8 x 8).  Residual RMS 0.57 in log; the
// intercept carries the 99th-percentile residual (+0.94) as a safety margin.
// Bytes = 2 levels x 20-byte records x prediction.
extern "C" uint64_t cc_serve_predict_bytes(uint32_t n, uint64_t m, uint32_t max_degree) {
  if (n < 4 || m < 4) return 4096;
  const double d = 2.0 * (double)m / (double)n;
  const double lp = kPredC[0] + kPredC[1] * n + kPredC[2] * d + kPredC[3] * max_degree + kPredC[4] * d * d;
  const double paths = std::exp(std::min(lp, 40.0));
  const double bytes = 2.0 * 20.0 * paths + 4096.0;
  return bytes > 1e18 ? (uint64_t)1e18 : (uint64_t)bytes;
}

// ------------------------------------------------------------------ lifecycle

extern "C" cc_status cc_serve_create(cc_context* c, const cc_serve_options* opts, cc_server** out) {
  if (!c || !out) return CC_ERR_ARG;
  *out = nullptr;
  cc_serve_options o{};
  if (opts) o = *opts;
  if (o.slots == 0) o.slots = 4096;
  if (o.slots > kMultiMaxSlots) return CC_ERR_UNSUPPORTED;
  if (o.admit_bytes == 0) o.admit_bytes = 64ull << 30;
  if (o.steps_per_round == 0) o.steps_per_round = 8;
  if (o.reserve_paths == 0) o.reserve_paths = 1ull << 18;
  cc_status s;
  if ((s = ensure_arena(c))) return s;
  if ((s = ensure_frames(c, 4096))) return s;
  cc_server* v = new cc_server();
  v->ctx = c;
  v->o = o;
  v->slots = o.slots;
  const unsigned int S = o.slots;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  const size_t o_adj = off; off = al(off + 8ull * 64 * S);
  const size_t o_rtab = off; off = al(off + 8ull * 64 * S);
  const size_t o_hist = off; off = al(off + 8ull * kHistW * S);
  const size_t o_tc = off; off = al(off + 8ull * kHistW * S);
  const size_t o_hash = off; off = al(off + 8ull * S);
  const size_t o_live = off; off = al(off + 8ull * S);
  const size_t o_Lg = off; off = al(off + S);
  const size_t o_dummy = off; off = al(off + 64);
  const size_t total = off;
  // upload staging: at most 1024 requests of n <= 64 per round
  v->up_bytes = al(4ull * 1024 * 65) + al(4ull * 1024 * 64 * 63) + al(8ull * 1025) * 2 + al(4ull * 1024) * 2;
  v->status_bytes = al(sizeof(Control)) + al(sizeof(Frame)) + 8ull * S;
  auto fail = [&](cc_status st) {
    cc_serve_destroy(v);
    return st;
  };
  if ((s = dev_alloc(c, (void**)&v->d_tab, total))) return fail(s);
  if ((s = dev_alloc(c, (void**)&v->d_up, v->up_bytes))) return fail(s);
  if ((s = dev_alloc(c, (void**)&v->d_out, 8ull * kOutW * S))) return fail(s);
  if ((s = dev_alloc(c, (void**)&v->d_gslots, 4ull * S))) return fail(s);
  if (cudaMallocHost((void**)&v->h_up, v->up_bytes) != cudaSuccess ||
      cudaMallocHost((void**)&v->h_out, 8ull * kOutW * S) != cudaSuccess ||
      cudaMallocHost((void**)&v->h_gslots, 4ull * S) != cudaSuccess ||
      cudaMallocHost((void**)&v->h_status, v->status_bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(CC_ERR_OOM);
  }
  v->d_adj = reinterpret_cast<unsigned long long*>(v->d_tab + o_adj);
  v->d_rtab = reinterpret_cast<unsigned long long*>(v->d_tab + o_rtab);
  v->d_hist = reinterpret_cast<unsigned long long*>(v->d_tab + o_hist);
  v->d_tcount = reinterpret_cast<unsigned long long*>(v->d_tab + o_tc);
  v->d_hash = reinterpret_cast<unsigned long long*>(v->d_tab + o_hash);
  v->d_live = reinterpret_cast<long long*>(v->d_tab + o_live);
  v->d_Lg = v->d_tab + o_Lg;
  v->d_dummy = reinterpret_cast<unsigned long long*>(v->d_tab + o_dummy);
  cudaStream_t stm = c->stream;
  if (cudaMemsetAsync(v->d_tab, 0, total, stm) != cudaSuccess ||
      cudaMemsetAsync(c->ctl, 0, sizeof(Control), stm) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(CC_ERR_CUDA);
  }
  // an empty frontier: both stacks empty
  Control h{};
  h.top = c->arena_bytes;
  if (cudaMemcpyAsync(&c->ctl->top, &h.top, sizeof(h.top), cudaMemcpyHostToDevice, stm) != cudaSuccess ||
      cudaStreamSynchronize(stm) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(CC_ERR_CUDA);
  }
  v->st.resize(S);
  v->free_slots.reserve(S);
  for (unsigned int i = S; i-- > 0;) v->free_slots.push_back(i);
  EngineParams& p = v->p;
  p.arena = c->arena;
  p.arena_bytes = c->arena_bytes;
  p.ctl = c->ctl;
  p.frames = c->frames;
  p.max_depth = c->frames_cap;
  p.n = 64;
  p.L = 64;
  p.maxch = 63;
  p.adj = v->d_adj;
  p.rtab = v->d_rtab;
  p.Lg = v->d_Lg;
  p.hist = v->d_hist;
  p.hash = v->d_hash;
  p.tcount = v->d_tcount;
  p.live = v->d_live;
  p.spin_limit = c->opts.spin_limit ? c->opts.spin_limit : kDefaultSpin;
  p.pf = c->opts.paths_per_thread;
  p.fresh = 0;
  p.max_steps = o.steps_per_round;
  p.reserve = o.reserve_paths;
  v->block = c->opts.threads_per_block ? (int)c->opts.threads_per_block : 256;
  v->grid = engine_grid(c, Kind::Multi, v->block, 0);
  if (v->grid <= 0) return fail(CC_ERR_CUDA);
  *out = v;
  return CC_OK;
}

extern "C" void cc_serve_destroy(cc_server* v) {
  if (!v) return;
  cc_context* c = v->ctx;
  if (c && c->stream) cudaStreamSynchronize(c->stream);
  dev_free(c, v->d_tab);
  dev_free(c, v->d_up);
  dev_free(c, v->d_out);
  dev_free(c, v->d_gslots);
  if (c && c->stream) cudaStreamSynchronize(c->stream);
  if (v->h_up) cudaFreeHost(v->h_up);
  if (v->h_out) cudaFreeHost(v->h_out);
  if (v->h_gslots) cudaFreeHost(v->h_gslots);
  if (v->h_status) cudaFreeHost(v->h_status);
  (void)cudaGetLastError();
  delete v;
}

extern "C" cc_status cc_serve_submit(cc_server* v, uint32_t n, const uint32_t* row_ptr, const uint32_t* col_idx,
                                     uint64_t predicted_bytes, uint64_t* out_id) {
  if (!v || !out_id) return CC_ERR_ARG;
  if (n > kMultiMaxN) return CC_ERR_UNSUPPORTED;
  Request r;
  unsigned int md = 0;
  cc_status s = validate_csr(n, row_ptr, col_idx, r.cols, &md);
  if (s) return s;
  r.id = v->next_id++;
  r.n = n;
  r.rows.assign(row_ptr, row_ptr + n + 1);
  const uint64_t m = row_ptr[n] / 2;
  r.pred_bytes = predicted_bytes ? predicted_bytes : cc_serve_predict_bytes(n, m, md);
  r.seed_bound = md > 1 ? (uint64_t)(md - 1) * m / 2 : 0;
  r.maxch = md > 1 ? md - 1 : 1;
  r.t_submit = Clock::now();
  v->queue.push_back(std::move(r));
  *out_id = v->queue.back().id;
  return CC_OK;
}

// ------------------------------------------------------------------ one round

extern "C" cc_status cc_serve_step(cc_server* v, cc_completion* out, uint32_t cap, uint32_t* n_out,
                                   uint32_t* in_flight, uint32_t* queued) {
  if (!v || !n_out || (cap && !out)) return CC_ERR_ARG;
  cc_context* c = v->ctx;
  cudaStream_t stm = c->stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
  };
  const size_t o_frame = (sizeof(Control) + 255) & ~size_t(255);
  const size_t o_live = o_frame + ((sizeof(Frame) + 255) & ~size_t(255));
  Control ctl{};
  Frame top{};
  std::memcpy(&ctl, v->h_status, sizeof(Control));
  std::memcpy(&top, v->h_status + o_frame, sizeof(Frame));
  const long long* live = reinterpret_cast<const long long*>(v->h_status + o_live);
  if (v->launched && ctl.err) return ctl.err == kDevTimeout ? CC_ERR_TIMEOUT : CC_ERR_CAPACITY;
  if (!v->launched) {
    ctl.depth = 0;
    ctl.top = c->arena_bytes;
  }

  // 1. completions: busy slots with no path in flight
  unsigned int ng = 0;
  if (v->launched) {
    for (unsigned int sl = 0; sl < v->slots; ++sl)
      if (v->st[sl].busy && live[sl] == 0) v->h_gslots[ng++] = sl;
  }
  if (ng) {
    ok(cudaMemcpyAsync(v->d_gslots, v->h_gslots, 4ull * ng, cudaMemcpyHostToDevice, stm));
    ok(launch_serve_gather(v->d_gslots, ng, v->d_hist, v->d_tcount, v->d_hash, v->d_out, stm));
    ok(cudaMemcpyAsync(v->h_out, v->d_out, 8ull * kOutW * ng, cudaMemcpyDeviceToHost, stm));
    ok(cudaStreamSynchronize(stm));
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return CC_ERR_CUDA;
    }
    const auto now = Clock::now();
    for (unsigned int i = 0; i < ng; ++i) {
      const unsigned int sl = v->h_gslots[i];
      SlotState& ss = v->st[sl];
      cc_completion cp{};
      cp.id = ss.id;
      const unsigned long long* r = v->h_out + (size_t)i * kOutW;
      for (int k = 0; k < kHistW; ++k) {
        cp.hist[k] = r[k];
        cp.total += r[k];
        cp.paths += r[kHistW + k];
      }
      cp.hash = r[2 * kHistW];
      cp.wait_us = std::chrono::duration<double, std::micro>(ss.t_admit - ss.t_submit).count();
      cp.latency_us = std::chrono::duration<double, std::micro>(now - ss.t_submit).count();
      v->done.push_back(cp);
      v->pred_in_flight -= ss.pred_bytes;
      v->n_maxch[ss.maxch] -= 1;
      v->n_L[ss.L] -= 1;
      ss.busy = false;
      v->free_slots.push_back(sl);
      v->in_flight -= 1;
    }
  }

  // 2. admission (arrival order), into the top frame's free records or a new frame 0
  const bool empty = ctl.depth == 0;
  const unsigned long long room =
      empty ? std::min<unsigned long long>(c->arena_bytes / 2 / 21, 1ull << 26) : top.stride - top.count;
  std::vector<Request*> adm;
  unsigned long long seeds = 0, up_rows = 0, up_cols = 0;
  const size_t max_up_cols = (size_t)1024 * 64 * 63;
  while (adm.size() < v->queue.size() && adm.size() < v->free_slots.size() && adm.size() < 1024) {
    Request& r = v->queue[adm.size()];
    // the budget never blocks the only request (a request larger than the budget still runs)
    if (v->in_flight + adm.size() > 0 && v->pred_in_flight + r.pred_bytes > v->o.admit_bytes) break;
    if (seeds + r.seed_bound > room || up_cols + r.cols.size() > max_up_cols) break;
    seeds += r.seed_bound;
    up_rows += r.rows.size();
    up_cols += r.cols.size();
    v->pred_in_flight += r.pred_bytes;
    adm.push_back(&r);
  }
  const unsigned int na = (unsigned int)adm.size();
  if (na) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    unsigned char* h = v->h_up;
    const size_t o_rows = 0, o_cols = al(4 * up_rows), o_roff = o_cols + al(4 * up_cols),
                 o_coff = o_roff + al(8ull * (na + 1)), o_n = o_coff + al(8ull * (na + 1)), o_sl = o_n + al(4ull * na),
                 o_end = o_sl + al(4ull * na);
    uint32_t* rows = reinterpret_cast<uint32_t*>(h + o_rows);
    uint32_t* cols = reinterpret_cast<uint32_t*>(h + o_cols);
    unsigned long long* roff = reinterpret_cast<unsigned long long*>(h + o_roff);
    unsigned long long* coff = reinterpret_cast<unsigned long long*>(h + o_coff);
    uint32_t* ns = reinterpret_cast<uint32_t*>(h + o_n);
    uint32_t* sls = reinterpret_cast<uint32_t*>(h + o_sl);
    size_t ro = 0, co = 0;
    const auto now = Clock::now();
    for (unsigned int i = 0; i < na; ++i) {
      Request& r = *adm[i];
      roff[i] = ro;
      coff[i] = co;
      std::memcpy(rows + ro, r.rows.data(), 4 * r.rows.size());
      if (!r.cols.empty()) std::memcpy(cols + co, r.cols.data(), 4 * r.cols.size());
      ro += r.rows.size();
      co += r.cols.size();
      ns[i] = r.n;
      const unsigned int sl = v->free_slots.back();
      v->free_slots.pop_back();
      sls[i] = sl;
      SlotState& ss = v->st[sl];
      ss.busy = true;
      ss.id = r.id;
      ss.pred_bytes = r.pred_bytes;
      ss.t_submit = r.t_submit;
      ss.t_admit = now;
      ss.maxch = r.maxch;
      ss.L = std::max(3u, (v->o.max_len == 0 || v->o.max_len > r.n) ? r.n : v->o.max_len);
      v->n_maxch[ss.maxch] += 1;
      v->n_L[ss.L] += 1;
    }
    roff[na] = ro;
    coff[na] = co;
    ok(cudaMemcpyAsync(v->d_up, h, o_end, cudaMemcpyHostToDevice, stm));
    unsigned long long fbase, fstride;
    unsigned long long *cnt_ptr, *next_ptr;
    if (empty) {
      // a fresh frame 0 at the bottom of the arena for the admitted triplets
      const unsigned long long stride = round_up(seeds + v->o.reserve_paths, 8);
      Frame f{};
      f.base = 0;
      f.bytes = multi_region_bytes(stride);
      f.stride = stride;
      f.next = 0;
      f.ncl = kNoNext;
      Control nc = ctl;
      nc.depth = 1;
      nc.bot = f.bytes;
      nc.top = c->arena_bytes;
      ok(cudaMemcpyAsync(c->frames, &f, sizeof(Frame), cudaMemcpyHostToDevice, stm));
      ok(cudaMemcpyAsync(&c->ctl->depth, &nc.depth, sizeof(nc.depth), cudaMemcpyHostToDevice, stm));
      ok(cudaMemcpyAsync(&c->ctl->bot, &nc.bot, sizeof(nc.bot), cudaMemcpyHostToDevice, stm));
      ok(cudaMemcpyAsync(&c->ctl->top, &nc.top, sizeof(nc.top), cudaMemcpyHostToDevice, stm));
      ok(cudaStreamSynchronize(stm));  // the host structs above are stack memory
      fbase = 0;
      fstride = stride;
      cnt_ptr = &c->frames[0].count;
      next_ptr = &c->frames[0].next;
      ctl.depth = 1;
    } else {
      fbase = top.base;
      fstride = top.stride;
      cnt_ptr = &c->frames[ctl.depth - 1].count;
      next_ptr = top.cursor == 0 ? &c->frames[ctl.depth - 1].next : v->d_dummy;
    }
    unsigned char* d = v->d_up;
    ok(launch_label_seed_multi(reinterpret_cast<unsigned int*>(d + o_rows),
                               reinterpret_cast<unsigned long long*>(d + o_roff),
                               reinterpret_cast<unsigned int*>(d + o_cols),
                               reinterpret_cast<unsigned long long*>(d + o_coff),
                               reinterpret_cast<unsigned int*>(d + o_n), reinterpret_cast<unsigned int*>(d + o_sl), na,
                               0, v->o.max_len, v->p, fbase, fstride, cnt_ptr, next_ptr, stm));
    v->queue.erase(v->queue.begin(), v->queue.begin() + na);
    v->in_flight += na;
  }

  // 3. expansion steps over the shared frontier
  if (ctl.depth > 0 || na) {
    unsigned int mc = 1, mL = 4;
    for (unsigned int i = kMultiMaxN; i > 0; --i)
      if (v->n_maxch[i]) { mc = i; break; }
    for (unsigned int i = kMultiMaxN; i > 3; --i)
      if (v->n_L[i]) { mL = i; break; }
    v->p.maxch = mc;
    v->p.L = mL;
    ok(launch_engine(Kind::Multi, v->p, v->grid, v->block, 0, stm));
    v->launched = true;
  }
  if (v->launched) {
    // status for the next round: control block, paths in flight per slot, top frame
    ok(cudaMemcpyAsync(v->h_status, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost, stm));
    ok(cudaMemcpyAsync(v->h_status + o_live, v->d_live, 8ull * v->slots, cudaMemcpyDeviceToHost, stm));
    ok(cudaStreamSynchronize(stm));
    if (e == cudaSuccess) {
      Control h;
      std::memcpy(&h, v->h_status, sizeof(Control));
      if (h.depth > 0) {
        ok(cudaMemcpyAsync(v->h_status + o_frame, c->frames + (h.depth - 1), sizeof(Frame), cudaMemcpyDeviceToHost,
                           stm));
        ok(cudaStreamSynchronize(stm));
      }
    }
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return CC_ERR_CUDA;
  }
  unsigned int k = 0;
  while (k < cap && !v->done.empty()) {
    out[k++] = v->done.front();
    v->done.pop_front();
  }
  *n_out = k;
  if (in_flight) *in_flight = v->in_flight;
  if (queued) *queued = (unsigned int)v->queue.size();
  return CC_OK;
}
