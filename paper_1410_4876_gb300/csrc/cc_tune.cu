// Autotuner of the launch configuration (cc_tune, cc_tune_batch in include/cc.h).
//
// The enumeration's results do not depend on the launch configuration; its speed does,
// and differently per graph class.  The tuner times candidate configurations through the
// public calls themselves, in stages (each stage keeps the best of the previous one):
//   1. adjacency form: bitset or CSR (single graphs with n <= 256)
//   2. launch shape: threads per block x persistent blocks per SM
//   3. paths per thread per round (bitset and batch expansion)
//   4. cluster phase: off, or the largest level it expands; two-level steps on or off
//      (bitset single graphs)
// Every candidate's histogram and hash must equal those of the configuration the context
// had on entry, so a tuning run is also a consistency check of the launch variants.
// Results are cached per (device name, graph class) in a JSON-lines file.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cc_host.hpp"

using namespace cc;

namespace {

std::string device_name(int dev) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return "unknown";
  }
  return prop.name;
}

unsigned int pow2_at_least(unsigned long long x) {
  unsigned int b = 1;
  while (b < x && b < (1u << 31)) b <<= 1;
  return b;
}

// one JSON object per line; fields written and read by this file only
const char* kKeys[] = {"threads_per_block", "blocks_per_sm", "paths_per_thread", "small_phase_paths", "mode",
                       "flags"};

unsigned int* knob(cc_options& o, int i) {
  switch (i) {
    case 0: return &o.threads_per_block;
    case 1: return &o.blocks_per_sm;
    case 2: return &o.paths_per_thread;
    case 3: return &o.small_phase_paths;
    case 4: return &o.mode;
    default: return &o.flags;
  }
}

bool read_uint(const std::string& line, const char* key, unsigned int* v) {
  const std::string k = std::string("\"") + key + "\": ";
  const size_t p = line.find(k);
  if (p == std::string::npos) return false;
  unsigned long x = 0;
  if (std::sscanf(line.c_str() + p + k.size(), "%lu", &x) != 1) return false;
  *v = (unsigned int)x;
  return true;
}

bool cache_lookup(const char* path, const std::string& dev, const std::string& cls, cc_options& o, double* ms) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  const std::string want_dev = "\"device\": \"" + dev + "\"", want_cls = "\"class\": \"" + cls + "\"";
  bool found = false;
  char buf[1024];
  while (std::fgets(buf, sizeof buf, f)) {
    const std::string line(buf);
    if (line.find(want_dev) == std::string::npos || line.find(want_cls) == std::string::npos) continue;
    cc_options t = o;
    bool ok = true;
    for (int i = 0; i < 6 && ok; ++i) ok = read_uint(line, kKeys[i], knob(t, i));
    if (!ok) continue;
    const size_t p = line.find("\"ms\": ");
    double m = 0;
    if (p != std::string::npos) std::sscanf(line.c_str() + p + 6, "%lf", &m);
    o = t;  // the last matching line wins
    *ms = m;
    found = true;
  }
  std::fclose(f);
  return found;
}

void cache_append(const char* path, const std::string& dev, const std::string& cls, cc_options& o, double ms) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "{\"device\": \"%s\", \"class\": \"%s\"", dev.c_str(), cls.c_str());
  for (int i = 0; i < 6; ++i) std::fprintf(f, ", \"%s\": %u", kKeys[i], *knob(o, i));
  std::fprintf(f, ", \"ms\": %.6f}\n", ms);
  std::fclose(f);
}

// The staged search.  `run(o, &ms)` times one configuration (CC_OK, or an error that
// ends the search); `bitset(o)` tells whether o runs a bitset path (stages 3-4).
template <typename Run, typename IsBitset>
cc_status search(cc_options base, bool try_csr, bool single, Run&& run, IsBitset&& bitset, cc_tune_result* out) {
  unsigned int timed = 0;
  double best_ms = 0;
  cc_options best = base;
  cc_status s = run(best, &best_ms);
  if (s) return s;
  ++timed;
  out->ms_default = best_ms;
  auto consider = [&](const cc_options& o) -> cc_status {
    double ms = 0;
    const cc_status r = run(o, &ms);
    if (r) return r;
    ++timed;
    if (ms < best_ms) {
      best_ms = ms;
      best = o;
    }
    return CC_OK;
  };
  // 1. adjacency form
  if (try_csr) {
    cc_options o = best;
    o.mode = CC_MODE_CSR;
    if ((s = consider(o))) return s;
  }
  // 2. launch shape
  {
    const cc_options start = best;
    for (unsigned int tpb : {128u, 256u})
      for (unsigned int bps = 1; bps <= 4; ++bps) {
        cc_options o = start;
        o.threads_per_block = tpb;
        o.blocks_per_sm = bps;
        if ((s = consider(o))) return s;
      }
  }
  // 3. paths per thread
  if (bitset(best)) {
    const cc_options start = best;
    for (unsigned int pf = 1; pf <= 3; ++pf) {
      cc_options o = start;
      o.paths_per_thread = pf;
      if ((s = consider(o))) return s;
    }
  }
  // 4. cluster phase and two-level steps
  if (single && bitset(best)) {
    const cc_options start = best;
    {
      cc_options o = start;
      o.flags |= CC_FLAG_NO_CLUSTER_PHASE;
      if ((s = consider(o))) return s;
    }
    {
      cc_options o = start;
      o.flags ^= CC_FLAG_NO_FUSE;
      if ((s = consider(o))) return s;
    }
    for (unsigned int sp : {8192u, 131072u}) {
      cc_options o = start;
      o.flags &= ~CC_FLAG_NO_CLUSTER_PHASE;
      o.small_phase_paths = sp;
      if ((s = consider(o))) return s;
    }
  }
  out->best = best;
  out->ms_best = best_ms;
  out->candidates = timed;
  return CC_OK;
}

void set_class(cc_tune_result* out, const std::string& cls) {
  std::snprintf(out->graph_class, sizeof out->graph_class, "%s", cls.c_str());
}

}  // namespace

extern "C" cc_status cc_tune(cc_graph* g, uint32_t max_len, const char* cache_path, cc_tune_result* out) {
  if (!g || !out) return CC_ERR_ARG;
  std::memset(out, 0, sizeof *out);
  cc_context* c = g->ctx;
  const cc_options entry = c->opts;
  out->best = entry;
  const unsigned int n = g->n;
  const unsigned int L = (max_len == 0 || max_len > n) ? n : max_len;
  // class: adjacency available, n and mean degree buckets, L'
  const double mean_deg = n ? 2.0 * (double)g->m / n : 0.0;
  char cls[64];
  std::snprintf(cls, sizeof cls, "single:%s:n%u:d%.1f:L%s", g->W ? "bitset" : "csr", pow2_at_least(n),
                std::round(mean_deg * 2.0) / 2.0, L == n ? "all" : std::to_string(L).c_str());
  set_class(out, cls);
  const std::string dev = device_name(c->device);
  double ms_cached = 0;
  cc_options cached = entry;
  if (cache_lookup(cache_path, dev, cls, cached, &ms_cached)) {
    out->best = cached;
    out->ms_best = ms_cached;
    out->from_cache = 1;
    return CC_OK;
  }
  if (n < 3 || L < 3) return CC_OK;
  // reference results with the entry options
  std::vector<uint64_t> ref(L + 1), hist(L + 1);
  uint64_t ref_hash = 0, hash = 0;
  cc_status s = cc_enumerate(g, max_len, ref.data(), &ref_hash, nullptr, nullptr, nullptr);
  if (s) return s;
  auto run = [&](const cc_options& o, double* ms) -> cc_status {
    c->opts.threads_per_block = o.threads_per_block;
    c->opts.blocks_per_sm = o.blocks_per_sm;
    c->opts.mode = o.mode;
    c->opts.flags = o.flags;
    c->opts.paths_per_thread = o.paths_per_thread;
    c->opts.small_phase_paths = o.small_phase_paths;
    double best = 0;
    for (int r = 0; r < 4; ++r) {  // one warm-up (and graph capture), then the best of three
      cc_run_info info{};
      const cc_status e = cc_enumerate(g, max_len, hist.data(), &hash, nullptr, nullptr, &info);
      if (e) return e;
      if (hash != ref_hash || hist != ref) return CC_ERR_CUDA;  // a launch variant disagrees
      if (r == 1 || (r > 1 && info.ms_proc < best)) best = info.ms_proc;
    }
    *ms = best;
    return CC_OK;
  };
  auto is_bitset = [&](const cc_options& o) { return g->W != 0 && o.mode != CC_MODE_CSR; };
  s = search(entry, g->W != 0, true, run, is_bitset, out);
  c->opts = entry;
  if (s) return s;
  cache_append(cache_path, dev, cls, out->best, out->ms_best);
  return CC_OK;
}

extern "C" cc_status cc_tune_batch(cc_context* c, uint32_t count, const uint32_t* n, const uint64_t* row_off,
                                   const uint32_t* row_ptr, const uint64_t* col_off, const uint32_t* col_idx,
                                   uint32_t max_len, const char* cache_path, cc_tune_result* out) {
  if (!c || !out || !n || count == 0) return CC_ERR_ARG;
  std::memset(out, 0, sizeof *out);
  if (c->batch.active) return CC_ERR_ARG;
  const cc_options entry = c->opts;
  out->best = entry;
  unsigned int nmax = 0;
  for (uint32_t g = 0; g < count; ++g) nmax = std::max(nmax, n[g]);
  char cls[64];
  std::snprintf(cls, sizeof cls, "batch:g%u:n%u:L%s", pow2_at_least(count), pow2_at_least(nmax),
                max_len ? std::to_string(max_len).c_str() : "all");
  set_class(out, cls);
  const std::string dev = device_name(c->device);
  double ms_cached = 0;
  cc_options cached = entry;
  if (cache_lookup(cache_path, dev, cls, cached, &ms_cached)) {
    out->best = cached;
    out->ms_best = ms_cached;
    out->from_cache = 1;
    return CC_OK;
  }
  const uint32_t stride = kMultiHistStride;
  std::vector<uint64_t> ref_hist((size_t)count * stride), ref_hash(count), hist((size_t)count * stride), hash(count);
  auto one = [&](std::vector<uint64_t>& h, std::vector<uint64_t>& hs, double* ms) -> cc_status {
    cc_batch_id id = 0;
    cc_status e = cc_batch_submit(c, count, n, row_off, row_ptr, col_off, col_idx, max_len, &id);
    if (e) return e;
    cc_run_info info{};
    do {
      e = cc_batch_poll(c, id, 1000000, h.data(), stride, hs.data(), nullptr, nullptr, &info);
    } while (e == CC_PENDING);
    if (ms) *ms = info.ms_proc;
    return e;
  };
  cc_status s = one(ref_hist, ref_hash, nullptr);
  if (s) return s;
  auto run = [&](const cc_options& o, double* ms) -> cc_status {
    c->opts.threads_per_block = o.threads_per_block;
    c->opts.blocks_per_sm = o.blocks_per_sm;
    c->opts.paths_per_thread = o.paths_per_thread;
    double t0 = 0, t1 = 0;
    cc_status e = one(hist, hash, &t0);  // warm-up
    if (e) return e;
    if (hist != ref_hist || hash != ref_hash) return CC_ERR_CUDA;
    if ((e = one(hist, hash, &t1))) return e;
    if (hist != ref_hist || hash != ref_hash) return CC_ERR_CUDA;
    *ms = t1;
    return CC_OK;
  };
  auto is_bitset = [](const cc_options&) { return true; };
  s = search(entry, false, false, run, is_bitset, out);
  c->opts = entry;
  if (s) return s;
  cache_append(cache_path, dev, cls, out->best, out->ms_best);
  return CC_OK;
}
