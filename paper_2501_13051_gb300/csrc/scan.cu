// Exclusive scan of uint32 counts into uint64 offsets (Algorithm 1's
// pos_buf) by reduce-then-scan: per-tile sums, one block scanning the tile
// sums, then a per-tile scan seeded with the tile's prefix.  No inter-block
// waiting, so no kernel here can stall on another block.
#include "kernels.h"

namespace cdl {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
static_assert(kScanTile == kScanThreads * kScanItems, "scan tile");
constexpr int kTopThreads = 1024;

__host__ __device__ constexpr uint32_t pad_idx(uint32_t i) { return i + (i >> 5); }

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                              uint64_t n,
                                                              uint64_t* __restrict__ tile_sums,
                                                              const uint64_t* dn) {
  __shared__ uint64_t red[kScanThreads / 32 + 1];
  n = dev_size(dn, n);
  // tile 0 is written even for n == 0; blocks loop over the tiles
  const uint64_t ntiles = n ? (n + kScanTile - 1) / kScanTile : 1;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t base = tile * kScanTile;
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const uint64_t idx = base + (uint64_t)i * kScanThreads + threadIdx.x;
      if (idx < n) s += __ldg(in + idx);
    }
    uint64_t total;
    block_exclusive_sum<kScanThreads, uint64_t>(s, red, &total);  // ends with a barrier
    if (threadIdx.x == 0) tile_sums[tile] = total;
  }
}

// One block: exclusive scan of the tile sums of n items in place; total ->
// *d_total.
__global__ void __launch_bounds__(kTopThreads) k_scan_top(uint64_t* __restrict__ sums, uint64_t n,
                                                          uint64_t* __restrict__ d_total,
                                                          const uint64_t* dn) {
  __shared__ uint64_t red[kTopThreads / 32 + 1];
  const uint64_t ntiles = (dev_size(dn, n) + kScanTile - 1) / kScanTile;
  uint64_t carry = 0;
  for (uint64_t b = 0; b < ntiles; b += kTopThreads) {
    const uint64_t i = b + threadIdx.x;
    const uint64_t v = i < ntiles ? sums[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_exclusive_sum<kTopThreads, uint64_t>(v, red, &tot);
    if (i < ntiles) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* __restrict__ in,
                                                             uint64_t n,
                                                             const uint64_t* __restrict__ prefix,
                                                             uint64_t* __restrict__ out,
                                                             const uint64_t* dn) {
  __shared__ uint32_t s_in[pad_idx(kScanTile) + 1];
  __shared__ uint64_t red[kScanThreads / 32 + 1];
  n = dev_size(dn, n);
  for (uint64_t tile = blockIdx.x; tile * kScanTile < n; tile += gridDim.x) {
    const uint64_t base = tile * kScanTile;
    // striped, coalesced load into shared memory
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      const uint32_t l = i * kScanThreads + threadIdx.x;
      const uint64_t idx = base + l;
      s_in[pad_idx(l)] = idx < n ? __ldg(in + idx) : 0u;
    }
    __syncthreads();
    // blocked: thread t owns tile elements [t*ITEMS, (t+1)*ITEMS)
    uint32_t v[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      v[i] = s_in[pad_idx(threadIdx.x * kScanItems + i)];
      s += v[i];
    }
    uint64_t tot;
    uint64_t run = block_exclusive_sum<kScanThreads, uint64_t>(s, red, &tot) + prefix[tile];
    const uint64_t first = base + (uint64_t)threadIdx.x * kScanItems;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      if (first + i < n) out[first + i] = run;
      run += v[i];
    }
  }
}

// Small inputs: one block walks the whole array with a running carry, so
// the scan is one launch instead of three.
constexpr uint64_t kSmallScan = 1 << 16;

__global__ void __launch_bounds__(kTopThreads) k_scan_small(const uint32_t* __restrict__ in,
                                                            uint64_t n, uint64_t* __restrict__ out,
                                                            uint64_t* __restrict__ d_total,
                                                            const uint64_t* dn) {
  __shared__ uint64_t red[kTopThreads / 32 + 1];
  n = dev_size(dn, n);
  constexpr int kI = 4;
  uint64_t carry = 0;
  for (uint64_t b = 0; b < n; b += (uint64_t)kTopThreads * kI) {
    const uint64_t first = b + (uint64_t)threadIdx.x * kI;
    uint32_t v[kI];
    uint64_t s = 0;
#pragma unroll
    for (int q = 0; q < kI; ++q) {
      v[q] = first + q < n ? __ldg(in + first + q) : 0u;
      s += v[q];
    }
    uint64_t tot;
    uint64_t run = carry + block_exclusive_sum<kTopThreads, uint64_t>(s, red, &tot);
#pragma unroll
    for (int q = 0; q < kI; ++q) {
      if (first + q < n) out[first + q] = run;
      run += v[q];
    }
    carry += tot;
  }
  if (threadIdx.x == 0 && d_total) *d_total = carry;
}

}  // namespace

size_t scan_workspace(uint64_t n) {
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  return ((tiles + 1) * sizeof(uint64_t) + 255) & ~size_t(255);
}

cudaError_t exclusive_scan(Ctx& c, const uint32_t* in, uint64_t n, uint64_t* out,
                           uint64_t* d_total, void* ws, const uint64_t* dn) {
  if (n == 0) {
    if (d_total) return cudaMemsetAsync(d_total, 0, sizeof(uint64_t), c.st);
    return cudaSuccess;
  }
  if (n <= kSmallScan) return scan_finish(c, in, n, out, d_total, ws, dn);
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  uint64_t* sums = static_cast<uint64_t*>(ws);
  {
    ProfScope p(c, c.scan_cls, 4.0 * n);
    k_scan_reduce<<<dev_grid(tiles, dn), kScanThreads, 0, c.st>>>(in, n, sums, dn);
  }
  return scan_finish(c, in, n, out, d_total, ws, dn);
}

cudaError_t scan_finish(Ctx& c, const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* d_total,
                        void* ws, const uint64_t* dn) {
  if (n == 0) {
    if (d_total) return cudaMemsetAsync(d_total, 0, sizeof(uint64_t), c.st);
    return cudaSuccess;
  }
  ProfScope p(c, c.scan_cls, 4.0 * n + 8.0 * n);
  if (n <= kSmallScan) {  // tile sums, if any were stored, are not needed
    k_scan_small<<<1, kTopThreads, 0, c.st>>>(in, n, out, d_total, dn);
    return cudaGetLastError();
  }
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  uint64_t* sums = static_cast<uint64_t*>(ws);
  k_scan_top<<<1, kTopThreads, 0, c.st>>>(sums, n, d_total, dn);
  k_scan_apply<<<dev_grid(tiles, dn), kScanThreads, 0, c.st>>>(in, n, sums, out, dn);
  return cudaGetLastError();
}

}  // namespace cdl
