// Host implementation of the C ABI declared in include/cc.h.
//
// A call of cc_enumerate runs, on the context's stream and without host round trips:
//   label kernel  (degree labelling, Section 2; relabelled adjacency and hash table)
//   seed kernel   (initial triplets and triangles, Section 4.3 / Algorithm 2)
//   engine        (persistent cooperative kernel: every expansion level, Section 4.4 /
//                  Algorithms 3 and 4, with the bounded-frontier depth-first fallback)
// followed by one device-to-host copy of the histogram, hash, level counts and status.
#include <algorithm>
#include <chrono>
#include <functional>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>


#include "cc_host.hpp"

using namespace cc;

// ------------------------------------------------------------------ context

static bool options_valid(const cc_options& o) {
  if (o.threads_per_block && (o.threads_per_block < 64 || o.threads_per_block > 256 || o.threads_per_block % 32))
    return false;
  if (o.mode > CC_MODE_CSR || o.blocks_per_sm > 4 || o.paths_per_thread > 4 || o.reserved) return false;
  return true;
}

extern "C" cc_status cc_context_create(const cc_options* opts, cc_context** out) {
  if (!out) return CC_ERR_ARG;
  *out = nullptr;
  cc_options o{};
  if (opts) o = *opts;
  if (!options_valid(o)) return CC_ERR_ARG;
  int dev = 0;
  CC_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CC_CUDA(cudaGetDeviceProperties(&prop, dev));
  if (!prop.cooperativeLaunch) return CC_ERR_CUDA;
  cc_context* c = new cc_context();
  c->device = dev;
  c->sms = prop.multiProcessorCount;
  c->opts = o;
  if (o.stream) {
    c->stream = static_cast<cudaStream_t>(o.stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return CC_ERR_CUDA;
    }
    c->own_stream = true;
  }
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    unsigned long long thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (dev_alloc(c, (void**)&c->ctl, sizeof(Control)) != CC_OK ||
      cudaMallocHost((void**)&c->h_ctl, sizeof(Control)) != cudaSuccess ||
      cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
      cudaEventCreate(&c->ev4) != cudaSuccess ||
      cudaEventCreate(&c->ev2) != cudaSuccess || cudaEventCreate(&c->ev3) != cudaSuccess) {
    (void)cudaGetLastError();
    cc_context_destroy(c);
    return CC_ERR_CUDA;
  }
  *out = c;
  return CC_OK;
}

extern "C" cc_status cc_context_set_options(cc_context* c, const cc_options* opts) {
  if (!c || !opts || !options_valid(*opts)) return CC_ERR_ARG;
  c->opts.threads_per_block = opts->threads_per_block;
  c->opts.blocks_per_sm = opts->blocks_per_sm;
  c->opts.mode = opts->mode;
  c->opts.spin_limit = opts->spin_limit;
  c->opts.flags = opts->flags;
  c->opts.paths_per_thread = opts->paths_per_thread;
  c->opts.small_phase_paths = opts->small_phase_paths;
  return CC_OK;
}

extern "C" void cc_context_destroy(cc_context* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  auto& b = c->batch;
  dev_free(c, b.d_pack);
  if (b.own) {
    dev_free(c, b.own->d_in);
    delete b.own;
  }
  dev_free(c, c->d_res);
  dev_free(c, c->d_trace);
  dev_free(c, c->frames);
  dev_free(c, c->ctl);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->own_arena && c->arena) cudaFree(c->arena);
  if (c->h_res) cudaFreeHost(c->h_res);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  if (c->h_stream) cudaFreeHost(c->h_stream);
  if (c->h_front) cudaFreeHost(c->h_front);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev2) cudaEventDestroy(c->ev2);
  if (c->ev3) cudaEventDestroy(c->ev3);
  if (c->ev4) cudaEventDestroy(c->ev4);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  (void)cudaGetLastError();
  delete c;
}

extern "C" const char* cc_status_str(cc_status s) {
  switch (s) {
    case CC_OK: return "ok";
    case CC_PENDING: return "pending";
    case CC_ERR_ARG: return "invalid argument";
    case CC_ERR_INVALID_GRAPH: return "not a simple undirected graph";
    case CC_ERR_OOM: return "out of memory";
    case CC_ERR_CUDA: return "CUDA error";
    case CC_ERR_TIMEOUT: return "device wait timed out";
    case CC_ERR_TRUNCATED: return "cycle list truncated";
    case CC_ERR_UNSUPPORTED: return "graph beyond supported limits";
    case CC_ERR_CAPACITY: return "frontier memory too small";
  }
  return "unknown status";
}

extern "C" void cc_get_limits(cc_limits* out) {
  if (!out) return;
  out->max_n_bitset = kBitsetMaxN;
  out->max_n_csr = kCsrMaxN;
  out->max_n_batch = kMultiMaxN;
  out->max_batch = kMultiMaxSlots;
}

// ------------------------------------------------------------------ graphs

extern "C" cc_status cc_graph_load(cc_context* c, uint32_t n, const uint32_t* row_ptr, const uint32_t* col_idx,
                                   cc_graph** out) {
  if (!c || !out) return CC_ERR_ARG;
  *out = nullptr;
  if (n > kCsrMaxN) return CC_ERR_UNSUPPORTED;
  std::vector<uint32_t> sorted;
  unsigned int md = 0;
  cc_status s = validate_csr(n, row_ptr, col_idx, sorted, &md);
  if (s) return s;
  cc_graph* g = new cc_graph();
  g->ctx = c;
  g->n = n;
  g->m = row_ptr[n] / 2;
  g->maxdeg = md;
  g->W = n <= 64 ? 1 : (n <= 128 ? 2 : (n <= 256 ? 4 : 0));
  const unsigned int npad = (n + 1) & ~1u;
  g->nrow_bytes = r16(4ull * (n + 1));
  g->ncol_bytes = r16(2ull * row_ptr[n]);
  g->rtab_bytes = r16(8ull * npad);
  g->adj_bytes = g->W ? r16(8ull * npad * g->W) : 0;
  g->nsig_bytes = r16(16ull * std::max<uint32_t>(n, 1));
  auto fail = [&](cc_status st) {
    cc_graph_free(g);
    return st;
  };
  // every buffer of the graph in one stream-ordered allocation (256-byte aligned parts):
  // the original CSR first, copied in one transfer, the rest zeroed by one memset
  auto a256 = [](unsigned long long x) { return (x + 255ull) & ~255ull; };
  const unsigned long long nnz = row_ptr[n];
  const unsigned long long o_row = 0, o_col = a256(4ull * (n + 1)), o_perm = a256(o_col + 4ull * std::max(nnz, 1ull));
  const unsigned long long o_rtab = a256(o_perm + 8ull * std::max<uint32_t>(n, 1)), o_nrow = a256(o_rtab + g->rtab_bytes);
  const unsigned long long o_ncol = a256(o_nrow + g->nrow_bytes), o_nsig = a256(o_ncol + g->ncol_bytes);
  const unsigned long long o_adj = a256(o_nsig + g->nsig_bytes), total = a256(o_adj + g->adj_bytes);
  if ((s = dev_alloc(c, (void**)&g->d_block, total))) return fail(s);
  unsigned char* b = g->d_block;
  g->d_row = reinterpret_cast<unsigned int*>(b + o_row);
  g->d_col = reinterpret_cast<unsigned int*>(b + o_col);
  g->d_perm = reinterpret_cast<unsigned int*>(b + o_perm);
  g->d_rtab = reinterpret_cast<unsigned long long*>(b + o_rtab);
  g->d_nrow = reinterpret_cast<unsigned int*>(b + o_nrow);
  g->d_ncol = reinterpret_cast<unsigned short*>(b + o_ncol);
  g->d_nsig = reinterpret_cast<unsigned long long*>(b + o_nsig);
  g->d_adj = g->W ? reinterpret_cast<unsigned long long*>(b + o_adj) : nullptr;
  // (from pageable memory: the call returns once the host copy is staged, so the vector
  // may go; the enumeration on the same stream sees the data)
  std::vector<uint32_t> up(o_col / 4 + nnz);
  std::memcpy(up.data(), row_ptr, 4ull * (n + 1));
  if (nnz) std::memcpy(up.data() + o_col / 4, sorted.data(), 4ull * nnz);
  if (cudaMemcpyAsync(b, up.data(), 4ull * up.size(), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemsetAsync(b + o_perm, 0, total - o_perm, c->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(CC_ERR_CUDA);
  }
  *out = g;
  return CC_OK;
}

extern "C" void cc_graph_free(cc_graph* g) {
  if (!g) return;
  cc_context* c = g->ctx;
  dev_free(c, g->d_block);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
}

extern "C" cc_status cc_graph_info(const cc_graph* g, uint32_t* n, uint64_t* m, uint32_t* max_degree) {
  if (!g) return CC_ERR_ARG;
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (max_degree) *max_degree = g->maxdeg;
  return CC_OK;
}

// ------------------------------------------------------------------ enumerate

namespace {
// A streamed cycle list (cc_enumerate_stream): device list capacities per round and the sink.
struct StreamOut {
  unsigned long long cap_c, cap_v;
  cc_cycle_sink sink;
  void* user;
  uint32_t rounds;
};

constexpr unsigned int kOffloadMinChunk = 4096;

// Bytes of n records of a frame of paths with t vertices, packed (stride n).
unsigned long long packed_bytes(Kind kind, int W, unsigned int t, unsigned long long n) {
  return is_csr(kind) ? n * 2ull * csr_rec_u16(t) : n * (8ull * W + 12ull);
}

// Copies the records [first, first + n) of a frame between its device region (plane
// stride f.stride) and a packed host block (plane stride n).
void copy_frame_records(unsigned char* arena, const Frame& f, Kind kind, int W, unsigned long long first,
                        unsigned long long n, unsigned char* host, bool to_host, cudaStream_t st,
                        const std::function<void(cudaError_t)>& ok) {
  auto cp = [&](unsigned long long dev_off, unsigned long long host_off, unsigned long long bytes) {
    if (to_host) ok(cudaMemcpyAsync(host + host_off, arena + dev_off, bytes, cudaMemcpyDeviceToHost, st));
    else ok(cudaMemcpyAsync(arena + dev_off, host + host_off, bytes, cudaMemcpyHostToDevice, st));
  };
  if (is_csr(kind)) {
    const unsigned long long rb = 2ull * csr_rec_u16(f.t);
    cp(f.base + first * rb, 0, n * rb);
    return;
  }
  for (int q = 0; q < W; ++q) cp(f.base + 8ull * (q * f.stride + first), 8ull * q * n, 8ull * n);  // B planes
  cp(f.base + 8ull * (W * f.stride + first), 8ull * W * n, 8ull * n);                              // H
  cp(f.base + 8ull * (W + 1) * f.stride + 4ull * first, 8ull * (W + 1) * n, 4ull * n);             // M
}

// The host-frontier loop of one enumeration (see cc_options.host_frontier_bytes).
cc_status host_frontier_loop(cc_context* c, Kind kind, int W, const EngineParams& p, int grid, int block, size_t smem,
                             cc_run_info& info, const std::function<void(cudaEvent_t)>& rec) {
  struct HostFrame {
    unsigned int t;
    unsigned long long n, next, ncl, off;
  };
  std::vector<HostFrame> hstack;
  unsigned long long hused = 0;
  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
  };
  if (!c->h_front) {
    if (cudaMallocHost((void**)&c->h_front, c->opts.host_frontier_bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      return CC_ERR_OOM;
    }
    c->h_front_bytes = c->opts.host_frontier_bytes;
  }
  std::vector<Frame> fr;
  for (;;) {
    Control& hc = *c->h_ctl;
    if (hc.err) return CC_OK;  // reported by the caller from the error word
    if (hc.want_offload) {
      // every device frame's unexpanded records to the host stack, bottom frame first
      fr.resize(hc.depth);
      ok(cudaMemcpyAsync(fr.data(), c->frames, sizeof(Frame) * hc.depth, cudaMemcpyDeviceToHost, st));
      ok(cudaStreamSynchronize(st));
      if (e != cudaSuccess) break;
      for (const Frame& f : fr) {
        const unsigned long long n = f.count > f.cursor ? f.count - f.cursor : 0ull;
        if (n == 0) continue;
        const unsigned long long bytes = packed_bytes(kind, W, f.t, n);
        if (hused + bytes > c->h_front_bytes) return CC_ERR_CAPACITY;
        copy_frame_records(c->arena, f, kind, W, f.cursor, n, c->h_front + hused, true, st, ok);
        hstack.push_back({f.t, n, f.cursor == 0 ? f.next : kNoNext, f.cursor == 0 ? f.ncl : kNoNext, hused});
        hused += (bytes + 255) & ~255ull;
      }
      ok(cudaStreamSynchronize(st));
      info.host_offloads += 1;
      hc.depth = 0;
    } else if (hc.depth != 0 || hstack.empty()) {
      break;  // finished (or stopped for another reason, reported by the caller)
    }
    if (hstack.empty()) break;
    // the most recent host frame back, alone, at the bottom of the arena
    const HostFrame hf = hstack.back();
    hstack.pop_back();
    hused = hf.off;
    Frame f{};
    f.base = 0;
    f.stride = round_up(hf.n, 8);
    f.bytes = is_csr(kind) ? csr_region_bytes(f.stride, hf.t) : bitset_region_bytes(f.stride, W);
    f.count = hf.n;
    f.cursor = 0;
    f.next = hf.next;
    f.ncl = hf.ncl;
    f.t = hf.t;
    f.end = 0;
    copy_frame_records(c->arena, f, kind, W, 0, hf.n, c->h_front + hf.off, false, st, ok);
    hc.depth = 1;
    hc.bot = f.bytes;
    hc.top = c->arena_bytes;
    hc.want_offload = 0;
    // (the frame from pageable memory is staged before the call returns; the control block
    // is the pinned mirror, left untouched until the sync below)
    ok(cudaMemcpyAsync(c->frames, &f, sizeof(Frame), cudaMemcpyHostToDevice, st));
    ok(cudaMemcpyAsync(c->ctl, &hc, sizeof(Control), cudaMemcpyHostToDevice, st));
    EngineParams q = p;
    q.fresh = 0;
    ok(launch_engine(kind, q, grid, block, smem, st));
    info.launches += 1;
    rec(c->ev1);
    ok(cudaMemcpyAsync(c->h_res, c->d_res, c->d_res_words * 8, cudaMemcpyDeviceToHost, st));
    ok(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    rec(c->ev2);
    ok(cudaStreamSynchronize(st));
    if (e != cudaSuccess) break;
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_status(e);
  }
  return CC_OK;
}

cc_status enumerate_impl(cc_graph* g, uint32_t max_len, uint64_t* out_hist, uint64_t* out_hash, uint64_t* out_tcount,
                         cc_cycles* out_cycles, StreamOut* so, cc_run_info* out_info, uint32_t part = 0,
                         uint32_t nparts = 1) {
  if (!g || !out_hist || !out_hash) return CC_ERR_ARG;
  if (nparts == 0 || part >= nparts) return CC_ERR_ARG;
  if (out_cycles && ((out_cycles->capacity_cycles && !out_cycles->offsets) ||
                     (out_cycles->capacity_vertices && !out_cycles->vertices)))
    return CC_ERR_ARG;
  cc_context* c = g->ctx;
  const unsigned int n = g->n;
  const unsigned int L = (max_len == 0 || max_len > n) ? n : max_len;
  std::memset(out_hist, 0, sizeof(uint64_t) * (L + 1));
  if (out_tcount) std::memset(out_tcount, 0, sizeof(uint64_t) * (L + 1));
  *out_hash = 0;
  cc_run_info info{};
  if (out_cycles) out_cycles->count = out_cycles->total_vertices = 0;

  // path choice: the bitset path needs n <= 256; the cycle list needs ordered paths (CSR)
  Kind kind;
  const unsigned int mode = c->opts.mode;
  const bool listing = out_cycles || so;
  if (mode == CC_MODE_BITSET && (g->W == 0 || listing)) return CC_ERR_UNSUPPORTED;
  if (listing || mode == CC_MODE_CSR || g->W == 0)
    kind = L <= 17 ? Kind::Csr16 : (L <= 33 ? Kind::Csr32 : Kind::Csr);  // stored paths have < L' vertices
  else kind = g->W == 1 ? Kind::Bitset1 : (g->W == 2 ? Kind::Bitset2 : Kind::Bitset4);
  info.mode = is_csr(kind) ? CC_MODE_CSR : CC_MODE_BITSET;
  if (n < 3 || L < 3) {
    if (out_info) *out_info = info;
    c->last = info;
    return CC_OK;
  }
  cc_status s;
  if ((s = ensure_arena(c))) return s;
  if ((s = ensure_frames(c, L + 4))) return s;
  const size_t words = 2ull * (L + 1) + 2;
  if ((s = ensure_results(c, words))) return s;
  unsigned long long* d_hist = c->d_res;
  unsigned long long* d_tcount = c->d_res + (L + 1);
  unsigned long long* d_hash = c->d_res + 2 * (L + 1);

  // optional cycle list buffers
  unsigned int* d_cv = nullptr;
  unsigned long long* d_cs = nullptr;
  unsigned int* d_cl = nullptr;
  const unsigned long long capc = so ? so->cap_c : (out_cycles ? out_cycles->capacity_cycles : 0);
  const unsigned long long capv = so ? so->cap_v : (out_cycles ? out_cycles->capacity_vertices : 0);
  auto free_cyc = [&]() {
    dev_free(c, d_cv);
    dev_free(c, d_cs);
    dev_free(c, d_cl);
  };
  // (streamed lists: every round must have room for one path's worst case, maxch cycles of
  // up to L' vertices, and the first round for the triangles, at most (Delta - 1) m / 2)
  const unsigned long long maxch = std::max(1u, g->maxdeg > 0 ? g->maxdeg - 1 : 1u);
  const unsigned long long tri = g->maxdeg > 1 ? (unsigned long long)(g->maxdeg - 1) * g->m / 2 : 0;
  if (so && (capc < std::max(maxch, tri) || capv < std::max(maxch * (L + 1), 3 * tri))) return CC_ERR_ARG;
  if (so) {
    const size_t hb = 12 * capc + 4 * capv;
    if (c->h_stream_bytes < hb) {
      if (c->h_stream) cudaFreeHost(c->h_stream);
  if (c->h_front) cudaFreeHost(c->h_front);
      c->h_stream = nullptr;
      c->h_stream_bytes = 0;
      CC_CUDA(cudaMallocHost((void**)&c->h_stream, hb));
      c->h_stream_bytes = hb;
    }
  }
  if (listing) {
    if ((s = dev_alloc(c, (void**)&d_cv, 4 * std::max(capv, 1ull))) ||
        (s = dev_alloc(c, (void**)&d_cs, 8 * std::max(capc, 1ull))) ||
        (s = dev_alloc(c, (void**)&d_cl, 4 * std::max(capc, 1ull)))) {
      free_cyc();
      return s;
    }
  }

  const int W = kind == Kind::Bitset1 ? 1 : (kind == Kind::Bitset2 ? 2 : (kind == Kind::Bitset4 ? 4 : 0));
  EngineParams p{};
  p.arena = c->arena;
  p.arena_bytes = c->arena_bytes;
  p.ctl = c->ctl;
  p.frames = c->frames;
  p.max_depth = c->frames_cap;
  p.n = n;
  p.L = L;
  p.maxch = std::max(1u, g->maxdeg > 0 ? g->maxdeg - 1 : 1u);
  p.adj = g->d_adj;
  p.rtab = g->d_rtab;
  p.nrow = g->d_nrow;
  p.ncol = g->d_ncol;
  p.nsig = g->d_nsig;
  p.perm = g->d_perm;
  p.hist = d_hist;
  p.hash = d_hash;
  p.tcount = d_tcount;
  p.spin_limit = c->opts.spin_limit ? c->opts.spin_limit : kDefaultSpin;
  p.fresh = 1;
  p.pf = c->opts.paths_per_thread;
  p.fuse_ok = (!is_csr(kind) && !(c->opts.flags & CC_FLAG_NO_FUSE)) ? 1u : 0u;
  p.seed_entries = (unsigned int)(2 * g->m);
  p.part = part;
  p.nparts = nparts;
  // the host frontier takes over when a level would be expanded in chunks of fewer than
  // this many paths while frames wait below it
  const bool host_front = c->opts.host_frontier_bytes > 0 && !so;
  p.offload_min = host_front ? kOffloadMinChunk : 0u;
  if (!c->d_trace) {
    if ((s = dev_alloc(c, (void**)&c->d_trace, 16ull * kTraceCap))) {
      free_cyc();
      return s;
    }
    c->trace_cap = kTraceCap;
  }
  p.step_ts = c->d_trace;
  p.step_rec = c->d_trace + c->trace_cap;
  p.step_ts_cap = c->trace_cap;
  p.cyc_vert = d_cv;
  p.cyc_start = d_cs;
  p.cyc_len = d_cl;
  p.cyc_cap_c = capc;
  p.cyc_cap_v = capv;
  p.cyc_stream = so ? 1u : 0u;
  // frame 0 (initial triplets) sized by |T(G)| <= (Delta - 1) m / 2 (Section 2)
  unsigned long long tb = g->maxdeg > 1 ? (unsigned long long)(g->maxdeg - 1) * g->m / 2 + 8 : 8;
  const unsigned long long seed_stride = round_up(tb, 8);
  const unsigned long long seed_bytes =
      is_csr(kind) ? csr_region_bytes(seed_stride, 3) : bitset_region_bytes(seed_stride, W);
  if (seed_bytes > c->arena_bytes / 2) {
    free_cyc();
    return CC_ERR_CAPACITY;
  }
  p.seed_stride = seed_stride;
  p.seed_bytes = seed_bytes;
  // graph staging into shared memory
  size_t smem = 0;
  if (is_csr(kind)) {
    // rows, neighbours and neighbour signatures (the r-table is read only when a cycle
    // closes and stays in global memory)
    const size_t need = g->nrow_bytes + g->ncol_bytes + g->nsig_bytes;
    if (need <= 160 * 1024) {
      p.smem_graph = 1;
      p.row_bytes = (unsigned int)g->nrow_bytes;
      p.adj_bytes = (unsigned int)(g->nrow_bytes + g->ncol_bytes);
      p.nsig_bytes = (unsigned int)g->nsig_bytes;
      smem = need;
    }
  } else {
    p.smem_graph = 1;
    p.adj_bytes = (unsigned int)g->adj_bytes;
    p.rtab_bytes = (unsigned int)g->rtab_bytes;
    smem = g->adj_bytes + g->rtab_bytes;
  }
  const int block = c->opts.threads_per_block ? (int)c->opts.threads_per_block : 256;
  const int grid = engine_grid(c, kind, block, smem);
  if (grid <= 0) {
    free_cyc();
    return CC_ERR_CUDA;
  }
  info.grid_blocks = grid;

  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
    return e == cudaSuccess;
  };
  // small levels first on one thread-block cluster (hardware barrier between levels),
  // then the persistent grid resumes from the state it leaves
  // (by default only for sparse graphs: with more children per path the phase's per-lane
  // loops are slower than the persistent grid's flattened form)
  int cs = 0;
  if (!is_csr(kind) && !(c->opts.flags & CC_FLAG_NO_CLUSTER_PHASE) &&
      (c->opts.small_phase_paths != 0 || p.maxch <= kClusterSparseMaxch)) {
    const unsigned long long key = (unsigned long long)kind | ((unsigned long long)smem << 8);
    cs = -1;
    for (auto& kv : c->cluster_sizes)
      if (kv.first == key) cs = kv.second;
    if (cs < 0) {
      cs = small_cluster_size(kind, smem);
      c->cluster_sizes.push_back({key, cs});
    }
  }
  const unsigned long long handover =
      c->opts.small_phase_paths ? c->opts.small_phase_paths : 2ull * (cs > 0 ? cs : 0) * 1024;
  info.launches = 3 + (cs > 0 ? 1 : 0);
  // the device work of the call, in stream order.  While capturing, events are recorded
  // as external event nodes so that every replay records them (a plain record in a
  // capture only orders the captured work).
  bool capturing = false;
  auto rec = [&](cudaEvent_t ev) {
    ok(capturing ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal) : cudaEventRecord(ev, st));
  };
  auto issue = [&]() {
    EngineParams q = p;
    rec(c->ev0);
    ok(cudaMemsetAsync(c->ctl, 0, sizeof(Control), st));
    ok(cudaMemsetAsync(c->d_res, 0, words * 8, st));
    ok(launch_label_single(g->d_row, g->d_col, n, (unsigned int)(2 * g->m), W, g->d_perm, g->d_adj, g->d_rtab,
                           g->d_nrow, g->d_ncol, g->d_nsig, st));
    ok(launch_seed_single(kind, q, seed_stride, st));
    rec(c->ev3);
    if (cs > 0) {
      ok(launch_small_engine(kind, q, cs, smem, handover, st));
      q.fresh = 0;
    }
    ok(launch_engine(kind, q, grid, block, smem, st));
    rec(c->ev1);
    ok(cudaMemcpyAsync(c->h_res, c->d_res, words * 8, cudaMemcpyDeviceToHost, st));
    ok(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    rec(c->ev2);
  };
  // CUDA graph: the key covers everything the captured work depends on (a host frontier
  // makes the call's launches depend on the run, so it is not captured)
  const bool use_graph = !listing && !host_front && !(c->opts.flags & CC_FLAG_NO_GRAPH) && !g->no_graph;
  unsigned long long gkey = 0;
  if (use_graph) {
    const unsigned long long parts[] = {(unsigned long long)kind, (unsigned long long)grid, (unsigned long long)block,
                                        (unsigned long long)smem, (unsigned long long)cs, handover,
                                        (unsigned long long)words, (unsigned long long)(uintptr_t)c->h_res,
                                        (unsigned long long)(uintptr_t)c->h_ctl, (unsigned long long)(uintptr_t)st};
    gkey = fnv1a(&p, sizeof(p), fnv1a(parts, sizeof(parts)));
  }
  if (use_graph && g->exec && g->exec_key == gkey) {
    ok(cudaGraphLaunch(g->exec, st));
    info.replayed = 1;
  } else if (use_graph && g->seen_key != gkey) {
    // first call with this configuration: launch directly (a graph enumerated once
    // never pays for a capture)
    g->seen_key = gkey;
    issue();
  } else if (use_graph) {
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool captured = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (captured) {
      capturing = true;
      issue();
      capturing = false;
      const cudaError_t ce = cudaStreamEndCapture(st, &gr);
      captured = e == cudaSuccess && ce == cudaSuccess && gr &&
                 cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess;
      if (gr) cudaGraphDestroy(gr);
    }
    if (captured) {
      if (g->exec) cudaGraphExecDestroy(g->exec);
      g->exec = ex;
      g->exec_key = gkey;
      ok(cudaGraphLaunch(g->exec, st));
      info.replayed = 1;
    } else {
      // not capturable here: launch directly from now on
      (void)cudaGetLastError();
      e = cudaSuccess;
      g->no_graph = true;
      issue();
    }
  } else {
    issue();
  }
  ok(cudaStreamSynchronize(st));
  // host frontier: when the engine stops for want of device memory (want_offload), every
  // frame on the device moves to pinned host memory (only its unexpanded records, packed)
  // and the top one comes back alone at the bottom of the arena; when the device stack
  // empties, the next frame comes back from the host.  The engine resumes each time from
  // the state it left (Section 6 leaves such a host-GPU transport to future work).
  cc_status hs = CC_OK;
  if (host_front && e == cudaSuccess) hs = host_frontier_loop(c, kind, W, p, grid, block, smem, info, rec);

  cc_status ss = CC_OK;
  while (so && e == cudaSuccess) {
    const Control& hc = *c->h_ctl;
    so->rounds += 1;
    if (hc.err != 0) break;
    if (hc.cyc_count > capc || hc.cyc_verts > capv) {  // (the planner's bound prevents this)
      ss = CC_ERR_TRUNCATED;
      break;
    }
    const unsigned long long nc = hc.cyc_count, nv = hc.cyc_verts;
    if (nc) {
      uint64_t* hs = reinterpret_cast<uint64_t*>(c->h_stream);
      uint32_t* hl = reinterpret_cast<uint32_t*>(hs + capc);
      uint32_t* hv = hl + capc;
      ok(cudaMemcpyAsync(hs, d_cs, 8 * nc, cudaMemcpyDeviceToHost, st));
      ok(cudaMemcpyAsync(hl, d_cl, 4 * nc, cudaMemcpyDeviceToHost, st));
      ok(cudaMemcpyAsync(hv, d_cv, 4 * nv, cudaMemcpyDeviceToHost, st));
      ok(cudaStreamSynchronize(st));
      if (e != cudaSuccess) break;
      so->sink(so->user, nc, hs, hl, hv, nv);
    }
    if (hc.depth == 0) break;
    if (nc == 0 && so->rounds > 1 && hc.step == info.steps) {  // no progress (cannot happen)
      ss = CC_ERR_CAPACITY;
      break;
    }
    info.steps = hc.step;
    EngineParams q = p;
    q.fresh = 0;
    ok(cudaMemsetAsync(&c->ctl->cyc_count, 0, 2 * sizeof(unsigned long long), st));
    ok(launch_engine(kind, q, grid, block, smem, st));
    info.launches += 1;
    rec(c->ev1);
    ok(cudaMemcpyAsync(c->h_res, c->d_res, words * 8, cudaMemcpyDeviceToHost, st));
    ok(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
    rec(c->ev2);
    ok(cudaStreamSynchronize(st));
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    free_cyc();
    info.dev_error = -(int)e;  // a CUDA API error: its code, negated
    c->last = info;
    if (out_info) *out_info = info;
    return cuda_status(e);
  }
  float ms1 = 0, ms2 = 0, ms3 = 0;
  if (cudaEventElapsedTime(&ms1, c->ev0, c->ev1) != cudaSuccess ||
      cudaEventElapsedTime(&ms2, c->ev0, c->ev2) != cudaSuccess ||
      cudaEventElapsedTime(&ms3, c->ev3, c->ev1) != cudaSuccess)
    (void)cudaGetLastError();  // timings stay 0; never leave an error for the caller's next call
  info.ms_engine = ms3;
  const Control& h = *c->h_ctl;
  s = map_dev_err(h.err);
  if (s == CC_OK) s = ss;
  if (s == CC_OK) s = hs;
  std::memcpy(out_hist, c->h_res, sizeof(uint64_t) * (L + 1));
  if (out_tcount) std::memcpy(out_tcount, c->h_res + (L + 1), sizeof(uint64_t) * (L + 1));
  *out_hash = c->h_res[2 * (L + 1)];
  info.ms_proc = ms1;
  info.ms_total = ms2;
  c->last_t_start = h.t_start;
  info.steps = h.step;
  info.spilled = h.spilled;
  info.dev_error = h.err;
  info.dev_error_info = h.err_info;
  info.peak_bytes = h.peak;
  for (unsigned int k = 0; k <= L; ++k) {
    info.cycles += c->h_res[k];
    info.paths += c->h_res[L + 1 + k];
  }
  if (s == CC_OK && out_cycles) {
    out_cycles->count = h.cyc_count;
    out_cycles->total_vertices = h.cyc_verts;
    if (h.cyc_count > capc || h.cyc_verts > capv) {
      s = CC_ERR_TRUNCATED;
    } else if (h.cyc_count) {
      std::vector<uint32_t> hv(h.cyc_verts);
      std::vector<unsigned long long> hs(h.cyc_count);
      std::vector<uint32_t> hl(h.cyc_count);
      if (cudaMemcpyAsync(hv.data(), d_cv, 4 * h.cyc_verts, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(hs.data(), d_cs, 8 * h.cyc_count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(hl.data(), d_cl, 4 * h.cyc_count, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        s = CC_ERR_CUDA;
      } else {
        uint64_t o = 0;
        out_cycles->offsets[0] = 0;
        for (unsigned long long i = 0; i < h.cyc_count; ++i) {
          std::memcpy(out_cycles->vertices + o, hv.data() + hs[i], 4ull * hl[i]);
          o += hl[i];
          out_cycles->offsets[i + 1] = o;
        }
      }
    } else if (capc) {
      out_cycles->offsets[0] = 0;
    }
  }
  free_cyc();
  c->last = info;
  if (out_info) *out_info = info;
  return s;
}
}  // namespace

extern "C" cc_status cc_enumerate(cc_graph* g, uint32_t max_len, uint64_t* out_hist, uint64_t* out_hash,
                                  uint64_t* out_tcount, cc_cycles* out_cycles, cc_run_info* out_info) {
  return enumerate_impl(g, max_len, out_hist, out_hash, out_tcount, out_cycles, nullptr, out_info);
}

extern "C" cc_status cc_enumerate_part(cc_graph* g, uint32_t max_len, uint32_t part, uint32_t nparts,
                                       uint64_t* out_hist, uint64_t* out_hash, uint64_t* out_tcount,
                                       cc_cycles* out_cycles, cc_run_info* out_info) {
  return enumerate_impl(g, max_len, out_hist, out_hash, out_tcount, out_cycles, nullptr, out_info, part, nparts);
}

extern "C" cc_status cc_enumerate_stream(cc_graph* g, uint32_t max_len, uint64_t chunk_cycles,
                                         uint64_t chunk_vertices, cc_cycle_sink sink, void* user, uint64_t* out_hist,
                                         uint64_t* out_hash, uint64_t* out_tcount, uint32_t* out_rounds,
                                         cc_run_info* out_info) {
  if (!sink) return CC_ERR_ARG;
  StreamOut so{chunk_cycles, chunk_vertices, sink, user, 0};
  const cc_status s = enumerate_impl(g, max_len, out_hist, out_hash, out_tcount, nullptr, &so, out_info);
  if (out_rounds) *out_rounds = so.rounds;
  return s;
}

extern "C" cc_status cc_get_trace(cc_context* c, uint32_t cap, uint64_t* t_ns, uint64_t* expanded, uint64_t* n_steps) {
  if (!c || !n_steps || (cap && (!t_ns || !expanded))) return CC_ERR_ARG;
  *n_steps = c->last.steps;
  if (!c->d_trace || cap == 0) return CC_OK;
  const unsigned long long k = std::min<unsigned long long>({(unsigned long long)cap, c->last.steps,
                                                            (unsigned long long)c->trace_cap});
  if (k == 0) return CC_OK;
  if (cudaMemcpyAsync(t_ns, c->d_trace, 8 * k, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(expanded, c->d_trace + c->trace_cap, 8 * k, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return CC_ERR_CUDA;
  }
  for (unsigned long long i = 0; i < k; ++i) t_ns[i] -= c->last_t_start;
  return CC_OK;
}

// ------------------------------------------------------------------ batch

// Validate and pack `count` graphs, and copy them into the set's device buffer (grown on
// demand).  Returns with the copies finished, so the caller's arrays may be released.
static cc_status batch_load_into(cc_batch_set* bs, uint32_t count, const uint32_t* n, const uint64_t* row_off,
                                 const uint32_t* row_ptr, const uint64_t* col_off, const uint32_t* col_idx,
                                 uint32_t* bad) {
  cc_context* c = bs->ctx;
  if (!n || !row_off || !row_ptr || !col_off) return CC_ERR_ARG;
  if (count == 0) return CC_ERR_ARG;
  if (count > kMultiMaxSlots) return CC_ERR_UNSUPPORTED;
  std::vector<uint32_t> rows, cols, sorted;
  std::vector<unsigned long long> roff(count + 1), coff(count + 1);
  unsigned long long tb_total = 0;
  unsigned int maxch = 1;
  for (uint32_t g = 0; g < count; ++g) {
    if (n[g] > kMultiMaxN) {
      *bad = g;
      return CC_ERR_UNSUPPORTED;
    }
    const uint32_t* rp = row_ptr + row_off[g];
    unsigned int md = 0;
    cc_status s = validate_csr(n[g], rp, col_idx ? col_idx + col_off[g] : nullptr, sorted, &md);
    if (s) {
      *bad = g;
      return s;
    }
    roff[g] = rows.size();
    coff[g] = cols.size();
    rows.insert(rows.end(), rp, rp + n[g] + 1);
    cols.insert(cols.end(), sorted.begin(), sorted.end());
    const unsigned long long m = rp[n[g]] / 2;
    // |T(G)| <= (max degree - 1) m / 2 (Section 2): the seed region's bound
    if (md > 1) tb_total += (unsigned long long)(md - 1) * m / 2;
    maxch = std::max(maxch, md > 1 ? md - 1 : 1u);
  }
  roff[count] = rows.size();
  coff[count] = cols.size();
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  bs->o_rows = off; off = al(off + 4 * rows.size());
  bs->o_cols = off; off = al(off + 4 * std::max<size_t>(cols.size(), 1));
  bs->o_roff = off; off = al(off + 8 * (count + 1));
  bs->o_coff = off; off = al(off + 8 * (count + 1));
  bs->o_n = off; off = al(off + 4 * count);
  const size_t total = off;
  cc_status s;
  if (bs->d_in_bytes < total) {
    dev_free(c, bs->d_in);
    bs->d_in = nullptr;
    bs->d_in_bytes = 0;
    if ((s = dev_alloc(c, &bs->d_in, total))) return s;
    bs->d_in_bytes = total;
  }
  unsigned char* base = static_cast<unsigned char*>(bs->d_in);
  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
  };
  ok(cudaMemcpyAsync(base + bs->o_rows, rows.data(), 4 * rows.size(), cudaMemcpyHostToDevice, st));
  if (!cols.empty()) ok(cudaMemcpyAsync(base + bs->o_cols, cols.data(), 4 * cols.size(), cudaMemcpyHostToDevice, st));
  ok(cudaMemcpyAsync(base + bs->o_roff, roff.data(), 8 * (count + 1), cudaMemcpyHostToDevice, st));
  ok(cudaMemcpyAsync(base + bs->o_coff, coff.data(), 8 * (count + 1), cudaMemcpyHostToDevice, st));
  ok(cudaMemcpyAsync(base + bs->o_n, n, 4 * count, cudaMemcpyHostToDevice, st));
  // synchronise so the host copies can be released when this call returns
  ok(cudaStreamSynchronize(st));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_status(e);
  }
  bs->count = count;
  bs->n.assign(n, n + count);
  bs->tb_total = tb_total;
  bs->maxch = maxch;
  bs->h2d_bytes = 4 * rows.size() + 4 * cols.size() + 16ull * (count + 1) + 4ull * count;
  return CC_OK;
}

extern "C" cc_status cc_batch_load(cc_context* c, uint32_t count, const uint32_t* n, const uint64_t* row_off,
                                   const uint32_t* row_ptr, const uint64_t* col_off, const uint32_t* col_idx,
                                   cc_batch_set** out, uint32_t* bad_graph) {
  if (!c || !out) return CC_ERR_ARG;
  *out = nullptr;
  cc_batch_set* bs = new (std::nothrow) cc_batch_set;
  if (!bs) return CC_ERR_OOM;
  bs->ctx = c;
  uint32_t bad = 0;
  cc_status s = batch_load_into(bs, count, n, row_off, row_ptr, col_off, col_idx, &bad);
  if (s) {
    if (bad_graph) *bad_graph = bad;
    dev_free(c, bs->d_in);
    delete bs;
    return s;
  }
  *out = bs;
  return CC_OK;
}

extern "C" void cc_batch_free(cc_batch_set* bs) {
  if (!bs) return;
  cc_context* c = bs->ctx;
  // a batch of this set may still be running: free after the context's stream
  if (c->batch.active && c->batch.set == bs) {
    cudaStreamSynchronize(c->stream);
    c->batch.active = false;
  }
  dev_free(c, bs->d_in);
  (void)cudaGetLastError();
  delete bs;
}

// Labelling, seeding and one persistent expansion launch for every graph of a loaded set
// (asynchronous on the context's stream; cc_batch_poll collects the results).
static cc_status batch_run(cc_batch_set* bs, uint32_t max_len, cc_batch_id* out) {
  cc_context* c = bs->ctx;
  auto& b = c->batch;
  if (b.active) return CC_ERR_ARG;
  const unsigned int count = bs->count;
  cc_status s;
  if ((s = ensure_arena(c))) return s;
  if ((s = ensure_frames(c, 70))) return s;
  // per-step trace (end time and paths expanded of each step) in the context's trace buffer
  if (!c->d_trace) {
    if ((s = dev_alloc(c, (void**)&c->d_trace, 16ull * kTraceCap))) return s;
    c->trace_cap = kTraceCap;
  }
  b.ts_cap = c->trace_cap;
  // work pack: adj | rtab | Lg | hist | hash | tcount | last
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  const size_t o_adj = off; off = al(off + 8ull * 64 * count);
  const size_t o_rtab = off; off = al(off + 8ull * 64 * count);
  const size_t o_Lg = off; off = al(off + count);
  const size_t o_hist = off; off = al(off + 8ull * kMultiHistStride * count);
  const size_t o_hash = off; off = al(off + 8ull * count);
  const size_t o_tc = off; off = al(off + 8ull * kMultiHistStride * count);
  const size_t o_last = off; off = al(off + 4ull * count);
  const size_t total = off;
  if (b.d_pack_bytes < total) {
    dev_free(c, b.d_pack);
    b.d_pack = nullptr;
    b.d_pack_bytes = 0;
    if ((s = dev_alloc(c, &b.d_pack, total))) return s;
    b.d_pack_bytes = total;
  }
  unsigned char* base = static_cast<unsigned char*>(b.d_pack);
  unsigned char* in = static_cast<unsigned char*>(bs->d_in);
  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
  };
  EngineParams p{};
  p.arena = c->arena;
  p.arena_bytes = c->arena_bytes;
  p.ctl = c->ctl;
  p.frames = c->frames;
  p.max_depth = c->frames_cap;
  p.n = 64;
  // the deepest stored level of any graph bounds the levels a depth-first chunk must leave
  // room for (each graph's own L' is in Lg)
  unsigned int maxL = 3;
  for (unsigned int g = 0; g < count; ++g)
    maxL = std::max(maxL, (max_len == 0 || max_len > bs->n[g]) ? bs->n[g] : max_len);
  p.L = maxL;
  p.maxch = bs->maxch;
  p.adj = reinterpret_cast<unsigned long long*>(base + o_adj);
  p.rtab = reinterpret_cast<unsigned long long*>(base + o_rtab);
  p.Lg = base + o_Lg;
  p.hist = reinterpret_cast<unsigned long long*>(base + o_hist);
  p.hash = reinterpret_cast<unsigned long long*>(base + o_hash);
  p.tcount = reinterpret_cast<unsigned long long*>(base + o_tc);
  p.last_step = reinterpret_cast<unsigned int*>(base + o_last);
  p.step_ts = c->d_trace;
  p.step_rec = c->d_trace + c->trace_cap;
  p.step_ts_cap = b.ts_cap;
  p.spin_limit = c->opts.spin_limit ? c->opts.spin_limit : kDefaultSpin;
  p.fresh = 1;
  p.pf = c->opts.paths_per_thread;
  p.fuse_ok = (c->opts.flags & CC_FLAG_NO_FUSE) ? 0u : 1u;
  const unsigned long long seed_stride = round_up(bs->tb_total + 8, 8);
  const unsigned long long seed_bytes = multi_region_bytes(seed_stride);
  if (seed_bytes > c->arena_bytes / 2) return CC_ERR_CAPACITY;
  p.seed_stride = seed_stride;
  p.seed_bytes = seed_bytes;
  const int block = c->opts.threads_per_block ? (int)c->opts.threads_per_block : 256;
  const int grid = engine_grid(c, Kind::Multi, block, 0);
  if (grid <= 0) return CC_ERR_CUDA;
  ok(cudaEventRecord(c->ev0, st));
  ok(cudaMemsetAsync(base + o_hist, 0, total - o_hist, st));
  ok(cudaMemsetAsync(c->ctl, 0, sizeof(Control), st));
  ok(launch_label_seed_multi(reinterpret_cast<unsigned int*>(in + bs->o_rows),
                             reinterpret_cast<unsigned long long*>(in + bs->o_roff),
                             reinterpret_cast<unsigned int*>(in + bs->o_cols),
                             reinterpret_cast<unsigned long long*>(in + bs->o_coff),
                             reinterpret_cast<unsigned int*>(in + bs->o_n), nullptr, count, 0, max_len, p, 0,
                             seed_stride, &c->ctl->seed_count, &c->ctl->seed_next, st));
  ok(cudaEventRecord(c->ev1, st));
  ok(launch_engine(Kind::Multi, p, grid, block, 0, st));
  ok(cudaEventRecord(c->ev2, st));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_status(e);
  }
  b.active = true;
  b.set = bs;
  b.count = count;
  b.max_len = max_len;
  b.L.resize(count);
  for (unsigned int g = 0; g < count; ++g)
    b.L[g] = (max_len == 0 || max_len > bs->n[g]) ? bs->n[g] : max_len;
  b.d_hist = p.hist;
  b.d_hash = p.hash;
  b.d_tcount = p.tcount;
  b.d_last = p.last_step;
  b.d_ts = p.step_ts;
  b.grid = grid;
  b.id = c->next_batch++;
  *out = b.id;
  return CC_OK;
}

extern "C" cc_status cc_batch_run(cc_batch_set* bs, uint32_t max_len, cc_batch_id* out) {
  if (!bs || !out) return CC_ERR_ARG;
  return batch_run(bs, max_len, out);
}

extern "C" cc_status cc_batch_submit(cc_context* c, uint32_t count, const uint32_t* n, const uint64_t* row_off,
                                     const uint32_t* row_ptr, const uint64_t* col_off, const uint32_t* col_idx,
                                     uint32_t max_len, cc_batch_id* out) {
  if (!c || !out) return CC_ERR_ARG;
  if (c->batch.active) return CC_ERR_ARG;
  if (!c->batch.own) {
    c->batch.own = new (std::nothrow) cc_batch_set;
    if (!c->batch.own) return CC_ERR_OOM;
    c->batch.own->ctx = c;
  }
  uint32_t bad = 0;
  cc_status s = batch_load_into(c->batch.own, count, n, row_off, row_ptr, col_off, col_idx, &bad);
  if (s) {
    if (s == CC_ERR_INVALID_GRAPH || s == CC_ERR_UNSUPPORTED) *out = bad;
    return s;
  }
  return batch_run(c->batch.own, max_len, out);
}

extern "C" cc_status cc_batch_poll(cc_context* c, cc_batch_id id, uint32_t timeout_us, uint64_t* hist,
                                   uint32_t hist_stride, uint64_t* hash, uint64_t* paths, double* done_us,
                                   cc_run_info* info) {
  if (!c || !hist || !hash || hist_stride == 0) return CC_ERR_ARG;
  auto& b = c->batch;
  if (!b.active || b.id != id) return CC_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaEventQuery(c->ev2);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) {
      (void)cudaGetLastError();
      b.active = false;
      return CC_ERR_CUDA;
    }
    const auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0);
    if ((uint64_t)el.count() >= timeout_us) return CC_PENDING;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  const unsigned int count = b.count;
  std::vector<unsigned long long> hh(kMultiHistStride * (size_t)count), ht(kMultiHistStride * (size_t)count),
      hs(count), ts;
  std::vector<unsigned int> hl(count);
  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
  };
  ok(cudaEventRecord(c->ev3, st));  // result copies: ms_total - ms_proc
  ok(cudaMemcpyAsync(hh.data(), b.d_hist, 8 * hh.size(), cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(ht.data(), b.d_tcount, 8 * ht.size(), cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(hs.data(), b.d_hash, 8 * count, cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(hl.data(), b.d_last, 4 * count, cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  ok(cudaEventRecord(c->ev4, st));
  ok(cudaStreamSynchronize(st));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    b.active = false;
    return CC_ERR_CUDA;
  }
  const Control& h = *c->h_ctl;
  const unsigned long long nsteps = h.step;
  ts.resize(std::min<unsigned long long>(nsteps, b.ts_cap));
  if (!ts.empty()) {
    ok(cudaMemcpyAsync(ts.data(), b.d_ts, 8 * ts.size(), cudaMemcpyDeviceToHost, st));
    ok(cudaStreamSynchronize(st));
  }
  b.active = false;
  cc_status s = map_dev_err(h.err);
  float ms_seed = 0, ms_all = 0;
  cudaEventElapsedTime(&ms_seed, c->ev0, c->ev1);
  cudaEventElapsedTime(&ms_all, c->ev0, c->ev2);
  cc_run_info ri{};
  float ms_eng = 0;
  cudaEventElapsedTime(&ms_eng, c->ev1, c->ev2);
  (void)cudaGetLastError();  // a failed timing query leaves no error for the caller
  float ms_copy = 0;
  cudaEventElapsedTime(&ms_copy, c->ev3, c->ev4);
  (void)cudaGetLastError();
  ri.ms_proc = ms_all;
  ri.ms_total = ms_all + ms_copy;
  ri.ms_engine = ms_eng;
  ri.steps = nsteps;
  ri.spilled = h.spilled;
  ri.peak_bytes = h.peak;
  ri.mode = CC_MODE_BITSET;
  ri.grid_blocks = b.grid;
  ri.launches = 2;  // labelling + seeding of every graph, one persistent expansion
  // step timestamps are absolute (globaltimer), measured from the engine's start
  const double t_start_ns = (double)h.t_start;
  for (unsigned int g = 0; g < count; ++g) {
    const unsigned int Lg = b.L[g];
    for (unsigned int k = 0; k < hist_stride; ++k)
      hist[(size_t)g * hist_stride + k] = (k <= Lg && k < (unsigned)kMultiHistStride) ? hh[(size_t)g * kMultiHistStride + k] : 0;
    hash[g] = hs[g];
    unsigned long long pg = 0, cg = 0;
    for (int k = 0; k < kMultiHistStride; ++k) {
      pg += ht[(size_t)g * kMultiHistStride + k];
      cg += hh[(size_t)g * kMultiHistStride + k];
    }
    if (paths) paths[g] = pg;
    ri.paths += pg;
    ri.cycles += cg;
    if (done_us) {
      // a graph is finished at the end of the last step that expanded one of its paths
      // (hl = 1 + that step; graphs with no stored path finish with seeding: 0)
      const unsigned int ls = hl[g];
      done_us[g] = (ls > 0 && ls - 1 < ts.size()) ? ((double)ts[ls - 1] - t_start_ns) / 1000.0 : 0.0;
    }
  }
  if (info) *info = ri;
  c->last = ri;
  c->last_t_start = h.t_start;  // cc_get_trace after a batch: steps timed from its start
  return s;
}
