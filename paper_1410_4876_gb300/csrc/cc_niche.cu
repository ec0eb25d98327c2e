// Niche overlap graph of a food web (Section 5: the paper's first group of graphs are food
// webs, directed graphs that it turns into undirected niche overlap graphs before the
// enumeration, following Wilson and Watkins).  Arc x -> z of the food web means that x
// feeds on z; two distinct species overlap when they have a prey in common.
//
// Three kernels on bitset rows of W = ceil(n / 64) words:
//   1. predators: Pred(z) |= bit x for every arc x -> z (a warp per species over its
//      prey list, atomicOr);
//   2. overlap rows: Row(x) = OR over the prey z of x of Pred(z), without x itself (one
//      warp per species, lanes over the row's words), and the row's popcount;
//   3. after an exclusive scan of the counts on the host's side of the call (the offsets
//      are needed there anyway), each row is written out as sorted neighbour ids.
// Memory: 2 n W words of rows (n = 32768: 256 MiB) and the output ids, allocated on the
// context's stream for the call.
#include <algorithm>
#include <vector>

#include "cc_host.hpp"

namespace {

__global__ void __launch_bounds__(256) niche_pred_kernel(const unsigned int* __restrict__ prey_ptr,
                                                         const unsigned int* __restrict__ prey_idx, unsigned int n,
                                                         unsigned int W, unsigned long long* pred) {
  const unsigned int x = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (x >= n) return;
  for (unsigned int e = prey_ptr[x] + (threadIdx.x & 31); e < prey_ptr[x + 1]; e += 32) {
    const unsigned int z = prey_idx[e];
    atomicOr(&pred[(unsigned long long)z * W + (x >> 6)], 1ull << (x & 63));
  }
}

__global__ void __launch_bounds__(256) niche_rows_kernel(const unsigned int* __restrict__ prey_ptr,
                                                         const unsigned int* __restrict__ prey_idx, unsigned int n,
                                                         unsigned int W, const unsigned long long* __restrict__ pred,
                                                         unsigned long long* rows, unsigned int* count) {
  const unsigned int x = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const unsigned int lane = threadIdx.x & 31;
  if (x >= n) return;
  unsigned int c = 0;
  for (unsigned int k = lane; k < W; k += 32) {
    unsigned long long r = 0;
    for (unsigned int e = prey_ptr[x]; e < prey_ptr[x + 1]; ++e) r |= pred[(unsigned long long)prey_idx[e] * W + k];
    if (k == (x >> 6)) r &= ~(1ull << (x & 63));
    rows[(unsigned long long)x * W + k] = r;
    c += __popcll(r);
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if (lane == 0) count[x] = c;
}

__global__ void __launch_bounds__(256) niche_write_kernel(unsigned int n, unsigned int W,
                                                          const unsigned long long* __restrict__ rows,
                                                          const unsigned int* __restrict__ row_ptr, unsigned int* col) {
  const unsigned int x = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const unsigned int lane = threadIdx.x & 31;
  if (x >= n) return;
  unsigned int out = row_ptr[x];
  for (unsigned int k0 = 0; k0 < W; k0 += 32) {
    const unsigned int k = k0 + lane;
    const unsigned long long r = k < W ? rows[(unsigned long long)x * W + k] : 0ull;
    const unsigned int c = __popcll(r);
    unsigned int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    unsigned int pos = out + incl - c;
    unsigned long long b = r;
    while (b) {
      col[pos++] = 64u * k + __ffsll((long long)b) - 1;
      b &= b - 1;
    }
    out += __shfl_sync(0xffffffffu, incl, 31);
  }
}

}  // namespace

extern "C" cc_status cc_niche_overlap(cc_context* c, uint32_t n, const uint32_t* prey_ptr, const uint32_t* prey_idx,
                                      uint32_t* out_row_ptr, uint32_t* out_col, uint64_t col_capacity,
                                      uint64_t* out_nnz) {
  if (!c || !prey_ptr || !out_row_ptr || !out_nnz) return CC_ERR_ARG;
  if (n > kCsrMaxN) return CC_ERR_UNSUPPORTED;
  if (prey_ptr[0] != 0) return CC_ERR_INVALID_GRAPH;
  for (uint32_t v = 0; v < n; ++v)
    if (prey_ptr[v + 1] < prey_ptr[v]) return CC_ERR_INVALID_GRAPH;
  const uint32_t arcs = prey_ptr[n];
  if (arcs && !prey_idx) return CC_ERR_ARG;
  for (uint32_t e = 0; e < arcs; ++e)
    if (prey_idx[e] >= n) return CC_ERR_INVALID_GRAPH;
  *out_nnz = 0;
  out_row_ptr[0] = 0;
  if (n == 0) return CC_OK;
  const unsigned int W = (n + 63) / 64;
  auto a256 = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t o_ptr = 0, o_idx = a256(4ull * (n + 1)), o_pred = a256(o_idx + 4ull * std::max<uint32_t>(arcs, 1));
  const size_t o_rows = a256(o_pred + 8ull * n * W), o_cnt = a256(o_rows + 8ull * n * W);
  const size_t o_rp = a256(o_cnt + 4ull * n), total = a256(o_rp + 4ull * (n + 1));
  unsigned char* d = nullptr;
  cc_status s = dev_alloc(c, (void**)&d, total);
  if (s) return s;
  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
  };
  unsigned int* d_ptr = reinterpret_cast<unsigned int*>(d + o_ptr);
  unsigned int* d_idx = reinterpret_cast<unsigned int*>(d + o_idx);
  unsigned long long* d_pred = reinterpret_cast<unsigned long long*>(d + o_pred);
  unsigned long long* d_rows = reinterpret_cast<unsigned long long*>(d + o_rows);
  unsigned int* d_cnt = reinterpret_cast<unsigned int*>(d + o_cnt);
  unsigned int* d_rp = reinterpret_cast<unsigned int*>(d + o_rp);
  ok(cudaMemcpyAsync(d_ptr, prey_ptr, 4ull * (n + 1), cudaMemcpyHostToDevice, st));
  if (arcs) ok(cudaMemcpyAsync(d_idx, prey_idx, 4ull * arcs, cudaMemcpyHostToDevice, st));
  ok(cudaMemsetAsync(d_pred, 0, 8ull * n * W, st));
  const unsigned int blocks = (n + 7) / 8;  // a warp per species, 8 per block
  niche_pred_kernel<<<blocks, 256, 0, st>>>(d_ptr, d_idx, n, W, d_pred);
  ok(cudaGetLastError());
  niche_rows_kernel<<<blocks, 256, 0, st>>>(d_ptr, d_idx, n, W, d_pred, d_rows, d_cnt);
  ok(cudaGetLastError());
  std::vector<uint32_t> cnt(n);
  ok(cudaMemcpyAsync(cnt.data(), d_cnt, 4ull * n, cudaMemcpyDeviceToHost, st));
  ok(cudaStreamSynchronize(st));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    dev_free(c, d);
    return cuda_status(e);
  }
  unsigned long long nnz = 0;
  for (uint32_t v = 0; v < n; ++v) {
    out_row_ptr[v] = (uint32_t)nnz;
    nnz += cnt[v];
  }
  out_row_ptr[n] = (uint32_t)nnz;
  *out_nnz = nnz;
  if (nnz > col_capacity || (nnz && !out_col)) {
    dev_free(c, d);
    return CC_ERR_TRUNCATED;
  }
  unsigned int* d_col = nullptr;
  if (nnz) {
    if ((s = dev_alloc(c, (void**)&d_col, 4ull * nnz))) {
      dev_free(c, d);
      return s;
    }
    ok(cudaMemcpyAsync(d_rp, out_row_ptr, 4ull * (n + 1), cudaMemcpyHostToDevice, st));
    niche_write_kernel<<<blocks, 256, 0, st>>>(n, W, d_rows, d_rp, d_col);
    ok(cudaGetLastError());
    ok(cudaMemcpyAsync(out_col, d_col, 4ull * nnz, cudaMemcpyDeviceToHost, st));
    ok(cudaStreamSynchronize(st));
    dev_free(c, d_col);
  }
  dev_free(c, d);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cuda_status(e);
  }
  return CC_OK;
}
