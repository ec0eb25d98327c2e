// Host-side state of the C ABI (private to the library's translation units).
#pragma once
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/cc.h"
#include "cc_internal.cuh"

using namespace cc;

namespace {

constexpr unsigned int kDefaultSpin = 1u << 25;   // ~8 s of polling at 256 ns
constexpr unsigned long long kDefaultFrontierCap = 64ull << 30;
constexpr unsigned int kTraceCap = 1u << 16;  // steps recorded per call

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct cc_context {
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cc_options opts{};
  unsigned char* arena = nullptr;
  unsigned long long arena_bytes = 0;
  bool own_arena = false;
  Control* ctl = nullptr;
  Frame* frames = nullptr;
  unsigned int frames_cap = 0;
  // per-call result buffers (device) and their pinned host mirrors
  unsigned long long* d_res = nullptr;  // hist | tcount | hash, grown on demand
  size_t d_res_words = 0;
  unsigned long long* h_res = nullptr;
  size_t h_res_words = 0;
  Control* h_ctl = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr, ev4 = nullptr;
  unsigned long long* d_trace = nullptr;  // per-step end time | paths expanded (last call)
  unsigned int trace_cap = 0;
  cc_run_info last{};
  std::vector<std::pair<unsigned long long, int>> cluster_sizes;  // (kind | smem << 8) -> size
  unsigned long long last_t_start = 0;  // globaltimer at the start of the last expansion
  unsigned char* h_stream = nullptr;    // pinned drain buffer of streamed cycle lists
  size_t h_stream_bytes = 0;
  unsigned char* h_front = nullptr;     // pinned host frontier (cc_options.host_frontier_bytes)
  size_t h_front_bytes = 0;
  // batch state (one batch in flight per context)
  struct Batch {
    cc_batch_set* set = nullptr;  // the set being enumerated
    cc_batch_set* own = nullptr;  // the set cc_batch_submit loads into (reused)
    cc_batch_id id = 0;
    bool active = false;
    unsigned int count = 0;
    unsigned int max_len = 0;
    std::vector<unsigned int> L;  // L' per graph
    void* d_pack = nullptr;       // per-slot tables and results
    size_t d_pack_bytes = 0;
    unsigned long long* d_hist = nullptr;
    unsigned long long* d_hash = nullptr;
    unsigned long long* d_tcount = nullptr;
    unsigned int* d_last = nullptr;
    unsigned long long* d_ts = nullptr;
    unsigned int ts_cap = 0;
    cc_status status = CC_OK;
    int grid = 0;
  } batch;
  cc_batch_id next_batch = 1;
};

// A set of graphs resident on the device for batched enumeration (cc_batch_load).
struct cc_batch_set {
  cc_context* ctx = nullptr;
  unsigned int count = 0;
  std::vector<unsigned int> n;     // vertices per graph
  unsigned long long tb_total = 0; // bound on the initial triplets of all graphs
  unsigned int maxch = 1;          // bound on children per path (max degree - 1)
  void* d_in = nullptr;            // rows | cols | row offsets | col offsets | n
  size_t d_in_bytes = 0;
  size_t o_rows = 0, o_cols = 0, o_roff = 0, o_coff = 0, o_n = 0;
  unsigned long long h2d_bytes = 0;  // bytes copied by the last load
};

struct cc_graph {
  cc_context* ctx = nullptr;
  unsigned int n = 0;
  unsigned long long m = 0;
  unsigned int maxdeg = 0;
  unsigned int* d_row = nullptr;    // original CSR (sorted rows)
  unsigned int* d_col = nullptr;
  unsigned int* d_perm = nullptr;   // [2n]: new->orig, orig->new
  unsigned long long* d_adj = nullptr;  // bitset rows (n <= 256), W words per row
  int W = 0;
  unsigned long long* d_rtab = nullptr;
  unsigned int* d_nrow = nullptr;   // relabelled CSR
  unsigned short* d_ncol = nullptr;
  unsigned long long* d_nsig = nullptr;  // neighbour signatures of the relabelled CSR [2n]
  unsigned char* d_block = nullptr;      // one allocation holding every buffer above
  size_t nrow_bytes = 0, ncol_bytes = 0, adj_bytes = 0, rtab_bytes = 0, nsig_bytes = 0;
  // captured device work of cc_enumerate for one launch configuration (CUDA graph)
  cudaGraphExec_t exec = nullptr;
  unsigned long long exec_key = 0;
  unsigned long long seen_key = 0;  // configuration of the previous call (captured on repeat)
  bool no_graph = false;            // capture failed once: launch directly
};

// FNV-1a over bytes (keys of captured CUDA graphs)
inline unsigned long long fnv1a(const void* data, size_t bytes, unsigned long long h = 1469598103934665603ull) {
  const unsigned char* b = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < bytes; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

// ------------------------------------------------------------------ helpers

inline cc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return CC_OK;
  if (e == cudaErrorMemoryAllocation) return CC_ERR_OOM;
  return CC_ERR_CUDA;
}

#define CC_CUDA(call)                              \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      (void)cudaGetLastError();                    \
      return cuda_status(e_);                      \
    }                                              \
  } while (0)

inline unsigned long long r16(unsigned long long x) { return (x + 15) & ~15ull; }

inline cc_status dev_alloc(cc_context* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  CC_CUDA(cudaMallocAsync(p, bytes, c->stream));
  return CC_OK;
}
inline void dev_free(cc_context* c, void* p) {
  if (p) cudaFreeAsync(p, c->stream);
}

inline cc_status ensure_results(cc_context* c, size_t words) {
  if (c->d_res_words < words) {
    dev_free(c, c->d_res);
    c->d_res = nullptr;
    c->d_res_words = 0;
    cc_status s = dev_alloc(c, (void**)&c->d_res, words * 8);
    if (s) return s;
    c->d_res_words = words;
  }
  if (c->h_res_words < words) {
    if (c->h_res) cudaFreeHost(c->h_res);
    c->h_res = nullptr;
    c->h_res_words = 0;
    CC_CUDA(cudaMallocHost((void**)&c->h_res, words * 8));
    c->h_res_words = words;
  }
  return CC_OK;
}

inline cc_status ensure_frames(cc_context* c, unsigned int depth) {
  if (c->frames_cap >= depth) return CC_OK;
  dev_free(c, c->frames);
  c->frames = nullptr;
  c->frames_cap = 0;
  unsigned int cap = std::max(depth, 256u);
  cc_status s = dev_alloc(c, (void**)&c->frames, sizeof(Frame) * cap);
  if (s) return s;
  c->frames_cap = cap;
  return CC_OK;
}

inline cc_status ensure_arena(cc_context* c) {
  if (c->arena) return CC_OK;
  if (c->opts.workspace) {
    if ((reinterpret_cast<uintptr_t>(c->opts.workspace) & 255) || c->opts.workspace_bytes < (1u << 20))
      return CC_ERR_ARG;
    c->arena = static_cast<unsigned char*>(c->opts.workspace);
    c->arena_bytes = c->opts.workspace_bytes & ~255ull;
    c->own_arena = false;
    return CC_OK;
  }
  unsigned long long want = c->opts.frontier_bytes;
  if (want == 0) {
    size_t fr = 0, tot = 0;
    CC_CUDA(cudaMemGetInfo(&fr, &tot));
    want = std::min<unsigned long long>(kDefaultFrontierCap, (unsigned long long)(fr * 0.4));
  }
  want &= ~255ull;
  if (want < (1u << 16)) return CC_ERR_ARG;
  void* p = nullptr;
  CC_CUDA(cudaMalloc(&p, want));
  c->arena = static_cast<unsigned char*>(p);
  c->arena_bytes = want;
  c->own_arena = true;
  return CC_OK;
}

// The cluster phase runs by default for graphs with at most this many children per path
// (maximum degree - 1); cc_options.small_phase_paths != 0 turns it on for every bitset graph.
constexpr unsigned int kClusterSparseMaxch = 4;

inline int engine_grid(cc_context* c, Kind kind, int block, size_t smem) {
  int bps = 0;
  if (engine_occupancy(kind, block, smem, &bps) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  unsigned int want = c->opts.blocks_per_sm ? c->opts.blocks_per_sm : 4u;
  bps = std::min<int>(bps, (int)want);
  return bps * c->sms;
}

// Validate a CSR (Section 1: finite undirected simple graph) and return sorted rows.
inline cc_status validate_csr(unsigned int n, const uint32_t* row_ptr, const uint32_t* col,
                              std::vector<uint32_t>& sorted, unsigned int* maxdeg) {
  if (!row_ptr) return CC_ERR_ARG;
  if (row_ptr[0] != 0) return CC_ERR_INVALID_GRAPH;
  for (unsigned int v = 0; v < n; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return CC_ERR_INVALID_GRAPH;
  const uint32_t nnz = row_ptr[n];
  if (nnz && !col) return CC_ERR_ARG;
  sorted.assign(col, col + nnz);
  unsigned int md = 0;
  for (unsigned int v = 0; v < n; ++v) {
    auto b = sorted.begin() + row_ptr[v], e = sorted.begin() + row_ptr[v + 1];
    std::sort(b, e);
    for (auto it = b; it != e; ++it) {
      if (*it >= n || *it == v) return CC_ERR_INVALID_GRAPH;
      if (it != b && *it == *(it - 1)) return CC_ERR_INVALID_GRAPH;
    }
    md = std::max(md, (unsigned int)(row_ptr[v + 1] - row_ptr[v]));
  }
  for (unsigned int v = 0; v < n; ++v)
    for (uint32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      const uint32_t w = sorted[e];
      if (!std::binary_search(sorted.begin() + row_ptr[w], sorted.begin() + row_ptr[w + 1], v))
        return CC_ERR_INVALID_GRAPH;
    }
  *maxdeg = md;
  return CC_OK;
}

inline cc_status map_dev_err(int err) {
  switch (err) {
    case kDevOk: return CC_OK;
    case kDevTimeout: return CC_ERR_TIMEOUT;
    case kDevCapacity: return CC_ERR_CAPACITY;
    case kDevSeedCap: return CC_ERR_CAPACITY;
    default: return CC_ERR_CUDA;
  }
}

