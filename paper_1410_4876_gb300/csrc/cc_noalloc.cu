// cc_enumerate_noalloc: the enumeration of cc_enumerate for callers that must not
// allocate memory.
//
// Who needs it: code that runs where cudaMalloc / cudaFree are not allowed or not
// acceptable - a plugin or real-time loop whose host application forbids device
// allocations after start-up, a process whose device memory is entirely owned by another
// pool allocator, or a latency-critical path where an allocation's implicit device-wide
// synchronisation would stall other streams.  Such a caller passes its graph and output
// buffers (host memory) and a stream; every device buffer the enumeration needs comes
// from one fixed, file-scope device array (kScratchBytes) that exists on every GPU that
// loads this library until the process exits.
//
// Nothing here allocates: no cudaMalloc/cudaFree/cudaMallocAsync, no host heap.  The
// device address of the array is looked up once per device (cudaGetSymbolAddress, with
// that device current) on the first call made on that device, so the first call on a
// device should come before any stream capture.  The address stays valid for the life of
// the device's primary context: a cudaDeviceReset (or any reset of that context) can move
// the array, and calls after it would use a stale address, so a process that resets a
// device must not call this entry point on that device afterwards.  All calls share the
// array and it keeps the previous call's contents: everything that must start at zero is
// cleared by each call, and calls whose work overlaps on the GPU (other streams, other
// host threads) race on the array and must be serialised by the caller.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/cc.h"
#include "cc_internal.cuh"

using namespace cc;

namespace {

constexpr unsigned long long kScratchBytes = 64ull << 20;  // CC_NOALLOC_SCRATCH_BYTES
constexpr unsigned int kMaxN = 256;                        // CC_NOALLOC_MAX_N
constexpr int kMaxDevices = 64;

// Fixed layout of the array (byte offsets, each rounded up to 256 bytes).
constexpr unsigned long long A256(unsigned long long x) { return (x + 255) & ~255ull; }
constexpr unsigned int kMaxFrames = 264;
constexpr unsigned long long kOffCtl = 0;
constexpr unsigned long long kOffFrames = A256(sizeof(Control));
constexpr unsigned long long kOffRes = A256(kOffFrames + kMaxFrames * sizeof(Frame));  // hist|tcount|hash
constexpr unsigned long long kOffRow = A256(kOffRes + 8ull * (2 * (kMaxN + 1) + 1));
constexpr unsigned long long kOffCol = A256(kOffRow + 4ull * (kMaxN + 1));
// the neighbour region holds n (n - 1) ids, the most a simple graph has; check_csr_in_place
// rejects a row_ptr[n] above that before anything is read or copied
constexpr unsigned long long kMaxCol = (unsigned long long)kMaxN * (kMaxN - 1);
constexpr unsigned long long kOffPerm = A256(kOffCol + 4ull * kMaxCol);
constexpr unsigned long long kOffAdj = A256(kOffPerm + 8ull * kMaxN);
constexpr unsigned long long kOffRtab = A256(kOffAdj + 8ull * kMaxN * 4);
constexpr unsigned long long kOffNrow = A256(kOffRtab + 8ull * kMaxN);
constexpr unsigned long long kOffNcol = A256(kOffNrow + 4ull * (kMaxN + 4));
constexpr unsigned long long kOffArena = A256(kOffNcol + 2ull * kMaxN * kMaxN);

static_assert(kOffArena + (16ull << 20) < kScratchBytes, "scratch array too small for its layout");

__device__ __align__(256) static unsigned char g_scratch[kScratchBytes];

std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
cc_status scratch_for_current_device(unsigned char** out, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return CC_ERR_CUDA;
  }
  if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return CC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || ptr == nullptr) {
      (void)cudaGetLastError();
      return CC_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_scratch_addr[dev];
  return CC_OK;
}

// Checks a host CSR in place (sorted strictly increasing rows, ids < n, no self-loops,
// symmetric), without copying it.  The offsets are checked first (row_ptr[n] at most
// n (n - 1), which also bounds the neighbour region of the array, and every row inside
// [0, row_ptr[n]]), so col_idx is never read beyond row_ptr[n] entries.
cc_status check_csr_in_place(uint32_t n, const uint32_t* rp, const uint32_t* col, unsigned int* maxdeg) {
  if (rp[0] != 0) return CC_ERR_INVALID_GRAPH;
  if ((unsigned long long)rp[n] > (unsigned long long)n * (n > 0 ? n - 1 : 0) || rp[n] > kMaxCol)
    return CC_ERR_INVALID_GRAPH;
  for (uint32_t v = 0; v < n; ++v)
    if (rp[v + 1] < rp[v] || rp[v + 1] > rp[n]) return CC_ERR_INVALID_GRAPH;
  if (rp[n] && !col) return CC_ERR_ARG;
  unsigned int md = 0;
  for (uint32_t v = 0; v < n; ++v) {
    for (uint32_t e = rp[v]; e < rp[v + 1]; ++e) {
      if (col[e] >= n || col[e] == v) return CC_ERR_INVALID_GRAPH;
      if (e > rp[v] && col[e] <= col[e - 1]) return CC_ERR_INVALID_GRAPH;
    }
    md = std::max(md, rp[v + 1] - rp[v]);
  }
  for (uint32_t v = 0; v < n; ++v)
    for (uint32_t e = rp[v]; e < rp[v + 1]; ++e) {
      const uint32_t w = col[e];
      if (!std::binary_search(col + rp[w], col + rp[w + 1], v)) return CC_ERR_INVALID_GRAPH;
    }
  *maxdeg = md;
  return CC_OK;
}

}  // namespace

extern "C" cc_status cc_enumerate_noalloc(uint32_t n, const uint32_t* row_ptr, const uint32_t* col_idx,
                                          uint32_t max_len, void* stream, uint64_t* out_hist, uint64_t* out_hash,
                                          uint64_t* out_tcount) {
  if (!row_ptr || !out_hist || !out_hash) return CC_ERR_ARG;
  if (n > kMaxN) return CC_ERR_UNSUPPORTED;
  const unsigned int L = (max_len == 0 || max_len > n) ? n : max_len;
  std::memset(out_hist, 0, sizeof(uint64_t) * (L + 1));
  if (out_tcount) std::memset(out_tcount, 0, sizeof(uint64_t) * (L + 1));
  *out_hash = 0;
  unsigned int maxdeg = 0;
  cc_status s = check_csr_in_place(n, row_ptr, col_idx, &maxdeg);
  if (s) return s;
  if (n < 3 || L < 3) return CC_OK;

  unsigned char* base = nullptr;
  int sms = 0;
  if ((s = scratch_for_current_device(&base, &sms))) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned long long m = row_ptr[n] / 2;
  const int W = n <= 64 ? 1 : (n <= 128 ? 2 : 4);
  const Kind kind = W == 1 ? Kind::Bitset1 : (W == 2 ? Kind::Bitset2 : Kind::Bitset4);
  const unsigned int npad = (n + 1) & ~1u;

  EngineParams p{};
  p.arena = base + kOffArena;
  p.arena_bytes = (kScratchBytes - kOffArena) & ~255ull;
  p.ctl = reinterpret_cast<Control*>(base + kOffCtl);
  p.frames = reinterpret_cast<Frame*>(base + kOffFrames);
  p.max_depth = kMaxFrames;
  p.n = n;
  p.L = L;
  p.maxch = std::max(1u, maxdeg > 1 ? maxdeg - 1 : 1u);
  unsigned long long* res = reinterpret_cast<unsigned long long*>(base + kOffRes);
  p.hist = res;
  p.tcount = res + (L + 1);
  p.hash = res + 2 * (L + 1);
  unsigned int* d_row = reinterpret_cast<unsigned int*>(base + kOffRow);
  unsigned int* d_col = reinterpret_cast<unsigned int*>(base + kOffCol);
  unsigned int* d_perm = reinterpret_cast<unsigned int*>(base + kOffPerm);
  unsigned long long* d_adj = reinterpret_cast<unsigned long long*>(base + kOffAdj);
  unsigned long long* d_rtab = reinterpret_cast<unsigned long long*>(base + kOffRtab);
  unsigned int* d_nrow = reinterpret_cast<unsigned int*>(base + kOffNrow);
  unsigned short* d_ncol = reinterpret_cast<unsigned short*>(base + kOffNcol);
  p.adj = d_adj;
  p.rtab = d_rtab;
  p.nrow = d_nrow;
  p.ncol = d_ncol;
  p.perm = d_perm;
  p.spin_limit = 1u << 25;
  p.fresh = 1;
  p.seed_entries = (unsigned int)(2 * m);
  const unsigned long long tb = maxdeg > 1 ? (unsigned long long)(maxdeg - 1) * m / 2 + 8 : 8;
  p.seed_stride = round_up(tb, 8);
  p.seed_bytes = bitset_region_bytes(p.seed_stride, W);
  if (p.seed_bytes > p.arena_bytes / 2) return CC_ERR_CAPACITY;
  p.smem_graph = 1;
  p.adj_bytes = (unsigned int)round_up(8ull * npad * W, 16);
  p.rtab_bytes = (unsigned int)round_up(8ull * npad, 16);
  const size_t smem = p.adj_bytes + p.rtab_bytes;
  const int block = 256;
  int bps = 0;
  if (engine_occupancy(kind, block, smem, &bps) != cudaSuccess || bps <= 0) {
    (void)cudaGetLastError();
    return CC_ERR_CUDA;
  }
  const int grid = std::min(bps, 4) * sms;

  const size_t words = 2ull * (L + 1) + 1;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
  };
  // the array keeps the previous call's contents: clear what must start at zero
  ok(cudaMemsetAsync(p.ctl, 0, sizeof(Control), st));
  ok(cudaMemsetAsync(res, 0, words * 8, st));
  ok(cudaMemcpyAsync(d_row, row_ptr, 4ull * (n + 1), cudaMemcpyHostToDevice, st));
  if (row_ptr[n]) ok(cudaMemcpyAsync(d_col, col_idx, 4ull * row_ptr[n], cudaMemcpyHostToDevice, st));
  ok(cudaMemsetAsync(d_rtab, 0, p.rtab_bytes, st));
  ok(launch_label_single(d_row, d_col, n, row_ptr[n], W, d_perm, d_adj, d_rtab, d_nrow, d_ncol, nullptr, st));
  ok(launch_seed_single(kind, p, p.seed_stride, st));
  ok(launch_engine(kind, p, grid, block, smem, st));
  Control h;
  ok(cudaMemcpyAsync(&h, p.ctl, sizeof(Control), cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(out_hist, res, 8ull * (L + 1), cudaMemcpyDeviceToHost, st));
  if (out_tcount) ok(cudaMemcpyAsync(out_tcount, res + (L + 1), 8ull * (L + 1), cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(out_hash, res + 2 * (L + 1), 8, cudaMemcpyDeviceToHost, st));
  ok(cudaStreamSynchronize(st));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;
  }
  switch (h.err) {
    case kDevOk: return CC_OK;
    case kDevTimeout: return CC_ERR_TIMEOUT;
    case kDevCapacity:
    case kDevSeedCap: return CC_ERR_CAPACITY;
    default: return CC_ERR_CUDA;
  }
}
