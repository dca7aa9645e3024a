// Step (c): LSD radix sort of tuples stored as separate uint32 columns
// (Section 5: per-column storage lets tuples be radix-sorted instead of
// merge-sorted).  The key of a tuple is its columns concatenated, column 0
// most significant, each column trimmed to its significant bits; passes take
// `bits`-wide digits of that packed key from the least significant end, so a
// relation over ids < 2^18 sorts in ceil(36 / 8) = 5 passes instead of 8.
//
// Each pass: (1) every tile of 4096 (or 2048) tuples counts its digits in shared
// memory; (2) an exclusive scan over the digit-major [digit][tile] counts
// gives every (digit, tile) run its global start; (3) every tile ranks its
// tuples stably (warp-level match on the digit, warps in order) and writes
// them through a shared-memory staging buffer so each digit's run leaves as
// contiguous stores.  Stable passes from least to most significant digit give
// the lexicographic order.
#include "kernels.h"

namespace cdl {

namespace {

// T threads per block (512 or 256, the tuner's choice) and kRItems tuples
// per thread: a tile holds T * kRItems tuples.
constexpr int kRItems = 8;
static_assert(kRItems % 4 == 0, "the upsweep reads items in chunks of four");

struct PassP {
  uint32_t sh[kMaxK], mask[kMaxK], dsh[kMaxK];
};

template <int K>
__device__ __forceinline__ uint32_t digit_of(const uint32_t (&v)[K], const PassP& p) {
  uint32_t d = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) d |= ((v[k] >> p.sh[k]) & p.mask[k]) << p.dsh[k];
  return d;
}

template <int K, int BITS, int T>
__global__ void __launch_bounds__(T) k_radix_upsweep(ColsIn in, uint64_t n, PassP p,
                                                     uint32_t* __restrict__ tile_hist,
                                                     uint64_t ntiles, const uint64_t* dn,
                                                     uint64_t* d_cells) {
  constexpr int R = 1 << BITS;
  constexpr int kRT = T, kRTile = T * kRItems;
  if (dn) {  // device-given size: the blocks loop over the tiles it gives
    n = dev_size(dn, n);
    ntiles = (n + kRTile - 1) / kRTile;
    // the length of the digit-major counts the pass's scan covers
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_cells = (uint64_t)R * ntiles;
  }
  __shared__ uint32_t h[R];
  // the counts need no order: with every column at a 16-byte boundary a
  // thread reads its items as 16-byte chunks of four (kRItems / 4 per
  // column, every load in flight before the first use)
  bool vec = true;
#pragma unroll
  for (int k = 0; k < K; ++k) vec &= (reinterpret_cast<uintptr_t>(in.c[k]) & 15u) == 0;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (int i = threadIdx.x; i < R; i += kRT) h[i] = 0;
    __syncthreads();
    const uint64_t base = tile * kRTile;
    uint32_t v[kRItems][K];
    if (vec && base + kRTile <= n) {
      constexpr int kC = kRItems / 4;
#pragma unroll
      for (int c = 0; c < kC; ++c) {
        const uint64_t e0 = base + 4u * ((uint64_t)c * kRT + threadIdx.x);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          uint4 w = make_uint4(0u, 0u, 0u, 0u);
          if (p.mask[k]) w = __ldg(reinterpret_cast<const uint4*>(in.c[k] + e0));
          v[4 * c][k] = w.x;
          v[4 * c + 1][k] = w.y;
          v[4 * c + 2][k] = w.z;
          v[4 * c + 3][k] = w.w;
        }
      }
#pragma unroll
      for (int it = 0; it < kRItems; ++it) atomicAdd(&h[digit_of<K>(v[it], p)], 1u);
    } else {
#pragma unroll
      for (int it = 0; it < kRItems; ++it) {
        const uint64_t idx = base + (uint64_t)it * kRT + threadIdx.x;
#pragma unroll
        for (int k = 0; k < K; ++k) v[it][k] = (idx < n && p.mask[k]) ? __ldg(in.c[k] + idx) : 0u;
      }
#pragma unroll
      for (int it = 0; it < kRItems; ++it) {
        const uint64_t idx = base + (uint64_t)it * kRT + threadIdx.x;
        if (idx < n) atomicAdd(&h[digit_of<K>(v[it], p)], 1u);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += kRT) tile_hist[(uint64_t)i * ntiles + tile] = h[i];
    __syncthreads();
  }
}

// Three resident blocks of 512 threads (or six of 256) per SM: registers
// capped at 42, shared memory carved out to the maximum by the launcher.
template <int K, int BITS, int T>
__global__ void __launch_bounds__(T, 1536 / T) k_radix_scatter(ColsIn in, ColsOut out, uint64_t n,
                                                             PassP p,
                                                             const uint64_t* __restrict__ off,
                                                             uint64_t ntiles, const uint64_t* dn) {
  constexpr int R = 1 << BITS;
  constexpr int kRT = T, kRTile = T * kRItems, kRW = T / 32;
  if (dn) {  // device-given size: the blocks loop over the tiles it gives
    n = dev_size(dn, n);
    ntiles = (n + kRTile - 1) / kRTile;
  }
  constexpr int DPT = (R + kRT - 1) / kRT;
  __shared__ uint32_t wh[kRW][R];  // per-warp digit counts, then per-warp offsets
  __shared__ uint32_t tstart[R];   // tile-local start of each digit's run
  __shared__ uint64_t gstart[R];   // global start of this tile's run of each digit, less its
                                   // tile-local start (an item at tile position i goes to
                                   // gstart[d] + i)
  __shared__ uint32_t red[kRT / 32 + 1];
  extern __shared__ uint32_t stage[];  // K x kRTile
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  for (int i = threadIdx.x; i < kRW * R; i += kRT) (&wh[0][0])[i] = 0;
  __syncthreads();
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  const uint64_t base = tile * kRTile;
  const uint64_t wbase = base + (uint64_t)warp * 32 * kRItems;
  uint32_t v[kRItems][K];
  uint32_t rk[kRItems];
#pragma unroll
  for (int it = 0; it < kRItems; ++it) {
    const uint64_t idx = wbase + (uint64_t)it * 32 + lane;
#pragma unroll
    for (int k = 0; k < K; ++k) v[it][k] = idx < n ? __ldg(in.c[k] + idx) : 0u;
  }
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int it = 0; it < kRItems; ++it) {
    const uint64_t idx = wbase + (uint64_t)it * 32 + lane;
    const bool valid = idx < n;
    const uint32_t d = valid ? digit_of<K>(v[it], p) : (uint32_t)R;
    // lanes holding the same digit: the lowest one advances the warp's
    // count of that digit for all of them and hands out the old count
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t leader = (uint32_t)__ffs(peers) - 1u;
    uint32_t b = 0;
    if (valid && lane == leader) b = atomicAdd(&wh[warp][d], (uint32_t)__popc(peers));
    b = __shfl_sync(0xffffffffu, b, leader);
    rk[it] = b + __popc(peers & lt);
  }
  __syncthreads();
  // per digit: exclusive offsets across warps (warp order = input order)
  for (int d = threadIdx.x; d < R; d += kRT) {
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < kRW; ++w) {
      const uint32_t t = wh[w][d];
      wh[w][d] = s;
      s += t;
    }
    tstart[d] = s;
    gstart[d] = off ? off[(uint64_t)d * ntiles + tile] : 0ull;
  }
  __syncthreads();
  {  // tile-local digit starts: exclusive scan of the digit totals
    uint32_t loc[DPT];
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = threadIdx.x * DPT + q;
      loc[q] = d < R ? tstart[d] : 0u;
      s += loc[q];
    }
    uint32_t tot;
    uint32_t ex = block_exclusive_sum<kRT, uint32_t>(s, red, &tot);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = threadIdx.x * DPT + q;
      if (d < R) tstart[d] = ex;
      ex += loc[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kRItems; ++it) {
    const uint64_t idx = wbase + (uint64_t)it * 32 + lane;
    if (idx < n) {
      const uint32_t d = digit_of<K>(v[it], p);
      const uint32_t pos = tstart[d] + wh[warp][d] + rk[it];
#pragma unroll
      for (int k = 0; k < K; ++k) stage[k * kRTile + pos] = v[it][k];
    }
  }
  // one tile (off null): its sorted order is the output order, g = i
  for (int d = threadIdx.x; d < R; d += kRT) gstart[d] = off ? gstart[d] - tstart[d] : 0ull;
  __syncthreads();
  const uint32_t tile_n = (uint32_t)(n - base < (uint64_t)kRTile ? n - base : kRTile);
  for (uint32_t i = threadIdx.x; i < tile_n; i += kRT) {
    uint32_t t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = stage[k * kRTile + i];
    const uint32_t d = digit_of<K>(t, p);
    const uint64_t g = gstart[d] + i;
#pragma unroll
    for (int k = 0; k < K; ++k) out.c[k][g] = t[k];
  }
  __syncthreads();  // the next tile reuses the shared tables and the staging buffer
  }
}

__global__ void k_column_max(ColsIn in, uint32_t k, uint64_t n, uint32_t* d_max) {
  for (uint32_t c = 0; c < k; ++c) {
    uint32_t m = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
      m = max(m, __ldg(in.c[c] + i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane_id() == 0) atomicMax(d_max + c, m);
  }
}

template <int K, int BITS, int T>
cudaError_t sort_passes(Ctx& c, const RadixPlan& plan, ColsOut a, ColsOut b, uint64_t n, void* ws,
                        bool* in_b, const uint64_t* dn) {
  constexpr int R = 1 << BITS;
  constexpr int kRT = T, kRTile = T * kRItems;
  const uint64_t ntiles = (n + kRTile - 1) / kRTile;
  const uint64_t cells = (uint64_t)R * ntiles;
  uint32_t* hist = static_cast<uint32_t*>(ws);
  uint64_t* off = reinterpret_cast<uint64_t*>(static_cast<char*>(ws) +
                                              ((cells * 4 + 255) & ~uint64_t(255)));
  void* scan_ws = reinterpret_cast<char*>(off) + ((cells * 8 + 255) & ~uint64_t(255));
  uint64_t* d_cells = nullptr;  // device-sized: scan length (the upsweep writes it)
  if (dn) d_cells = reinterpret_cast<uint64_t*>(static_cast<char*>(scan_ws) + scan_workspace(cells));
  const size_t smem = sizeof(uint32_t) * K * kRTile;
  cudaError_t e = cudaFuncSetAttribute(k_radix_scatter<K, BITS, T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_radix_scatter<K, BITS, T>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  ColsOut src = a, dst = b;
  bool flip = false;
  for (uint32_t pi = 0; pi < plan.npass; ++pi) {
    PassP p;
    for (int k = 0; k < kMaxK; ++k) {
      p.sh[k] = plan.pass[pi].sh[k];
      p.mask[k] = plan.pass[pi].mask[k];
      p.dsh[k] = plan.pass[pi].dsh[k];
    }
    ColsIn in;
    for (int k = 0; k < kMaxK; ++k) in.c[k] = src.c[k];
    uint32_t cols_used = 0;
    for (int k = 0; k < K; ++k) cols_used += p.mask[k] != 0;
    // one tile: its own ranking is the global order, no histogram pass
    const bool single = ntiles == 1 && !dn;
    if (!single) {
      {
        ProfScope ps(c, kRadixUpsweep, 4.0 * cols_used * n + 4.0 * cells);
        k_radix_upsweep<K, BITS, T><<<dev_grid(ntiles, dn), kRT, 0, c.st>>>(in, n, p, hist, ntiles,
                                                                            dn, d_cells);
      }
      e = exclusive_scan(c, hist, cells, off, nullptr, scan_ws, d_cells);
      if (e != cudaSuccess) return e;
    }
    {
      ProfScope ps(c, kRadixScatter, 8.0 * K * n);
      k_radix_scatter<K, BITS, T><<<dev_grid(ntiles, dn), kRT, smem, c.st>>>(
          in, dst, n, p, single ? nullptr : off, ntiles, dn);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::swap(src, dst);
    flip = !flip;
  }
  *in_b = flip;
  return cudaSuccess;
}

template <int K>
cudaError_t sort_k(Ctx& c, const RadixPlan& plan, ColsOut a, ColsOut b, uint64_t n, void* ws,
                   bool* in_b, const uint64_t* dn) {
  const bool wide = plan.threads == 512;
  switch (plan.bits) {
    case 8:
      return wide ? sort_passes<K, 8, 512>(c, plan, a, b, n, ws, in_b, dn)
                  : sort_passes<K, 8, 256>(c, plan, a, b, n, ws, in_b, dn);
    case 9:
      return wide ? sort_passes<K, 9, 512>(c, plan, a, b, n, ws, in_b, dn)
                  : sort_passes<K, 9, 256>(c, plan, a, b, n, ws, in_b, dn);
    case 10:
      return wide ? sort_passes<K, 10, 512>(c, plan, a, b, n, ws, in_b, dn)
                  : sort_passes<K, 10, 256>(c, plan, a, b, n, ws, in_b, dn);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

uint32_t fit_digit_bits(uint32_t total_bits, uint32_t base) {
  if (base != 8) return base;
  const uint32_t p8 = (total_bits + 7) / 8;
  return (p8 > 1 && total_bits <= 9 * (p8 - 1)) ? 9u : 8u;
}

RadixPlan make_radix_plan(uint32_t k, const uint32_t* col_bits, uint32_t digit_bits,
                          uint32_t threads) {
  RadixPlan pl;
  pl.k = k;
  pl.bits = (digit_bits == 10 || digit_bits == 9) ? digit_bits : 8;
  pl.threads = threads == 256 ? 256 : 512;
  uint32_t pos[kMaxK] = {0, 0, 0, 0};
  uint32_t total = 0;
  for (int c = (int)k - 1; c >= 0; --c) {
    pos[c] = total;
    total += col_bits[c];
  }
  pl.npass = (total + pl.bits - 1) / pl.bits;
  for (uint32_t p = 0; p < pl.npass; ++p) {
    RadixPlan::Pass ps{};
    const uint32_t lo = p * pl.bits, hi = lo + pl.bits < total ? lo + pl.bits : total;
    for (uint32_t c = 0; c < k; ++c) {
      const uint32_t s = lo > pos[c] ? lo : pos[c];
      const uint32_t e = hi < pos[c] + col_bits[c] ? hi : pos[c] + col_bits[c];
      if (s < e) {
        ps.sh[c] = s - pos[c];
        ps.mask[c] = (e - s >= 32) ? 0xFFFFFFFFu : ((1u << (e - s)) - 1u);
        ps.dsh[c] = s - lo;
      }
    }
    pl.pass.push_back(ps);
  }
  return pl;
}

size_t radix_workspace(uint64_t n, uint32_t digit_bits, uint32_t threads) {
  const uint64_t R = 1ull << ((digit_bits == 10 || digit_bits == 9) ? digit_bits : 8);
  const uint64_t tile = (threads == 256 ? 256 : 512) * kRItems;
  const uint64_t ntiles = (n + tile - 1) / tile;
  const uint64_t cells = R * ntiles;
  return ((cells * 4 + 255) & ~uint64_t(255)) + ((cells * 8 + 255) & ~uint64_t(255)) +
         scan_workspace(cells) + 256;
}

cudaError_t radix_sort(Ctx& c, const RadixPlan& plan, ColsOut a, ColsOut b, uint64_t n, void* ws,
                       bool* in_b, const uint64_t* dn) {
  *in_b = false;
  if ((n <= 1 && !dn) || n == 0 || plan.npass == 0) return cudaSuccess;
  switch (plan.k) {
    case 1: return sort_k<1>(c, plan, a, b, n, ws, in_b, dn);
    case 2: return sort_k<2>(c, plan, a, b, n, ws, in_b, dn);
    case 3: return sort_k<3>(c, plan, a, b, n, ws, in_b, dn);
    case 4: return sort_k<4>(c, plan, a, b, n, ws, in_b, dn);
    case 5: return sort_k<5>(c, plan, a, b, n, ws, in_b, dn);
    case 6: return sort_k<6>(c, plan, a, b, n, ws, in_b, dn);
    case 7: return sort_k<7>(c, plan, a, b, n, ws, in_b, dn);
    case 8: return sort_k<8>(c, plan, a, b, n, ws, in_b, dn);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t column_max(Ctx& c, ColsIn in, uint32_t k, uint64_t n, uint32_t* d_max) {
  cudaError_t e = cudaMemsetAsync(d_max, 0, sizeof(uint32_t) * k, c.st);
  if (e != cudaSuccess || n == 0) return e;
  ProfScope ps(c, kMisc, 4.0 * k * n);
  uint64_t blocks = (n + 2047) / 2048;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_column_max<<<(unsigned)blocks, 256, 0, c.st>>>(in, k, n, d_max);
  return cudaGetLastError();
}

}  // namespace cdl
