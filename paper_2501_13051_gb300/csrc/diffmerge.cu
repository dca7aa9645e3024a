// Step (d): set difference + eager merge (Section 4, "Union and
// Deduplication": delta = New - Full by the difference operator; Section 3,
// "Continuous Memory Layout": delta merged at once into one contiguous,
// sorted Full).  Both inputs are sorted; Full is unique, New may repeat.  In
// the merged order a Full tuple precedes an equal New tuple, so a New tuple
// is a repeat exactly when it equals the Full tuple or the New tuple just
// before it in that order: the removal of repeats (step c's "unique") is
// folded into this step.
//
// The combined sequence is cut into tiles of 4096 items by merge-path splits
// (Green, McColl & Bader, "GPU merge path", ICS 2012), computed for all
// tiles at once by a small kernel with one thread per split.  Then:
//   count  -- per tile, every New tuple finds its co-rank in the tile's Full
//             slice (how many of its Full tuples are <= it) and whether it
//             repeats a Full tuple.  A tile whose New tuples are at least a
//             quarter of its Full ones stages both slices in shared memory
//             and merges them again, each thread walking 16 items from its
//             own merge-path split; one with fewer (but at least a
//             sixteenth) stages its Full slice and searches it per New
//             tuple; a sparse one
//             binary-searches its Full slice with cached global loads, two
//             searches per thread stepping together, and touches few Full
//             sectors.  The co-rank of every New tuple (or a repeat mark)
//             and the tile's count of new tuples are stored;
//   scan   -- exclusive scan of the tile counts: each tile's delta offset
//             and |delta|;
//   write  -- per tile, a block scan ranks its new tuples, a histogram of
//             their co-ranks scanned over the Full slice gives every Full
//             tuple its shift (the new tuples placed before it), and the
//             Full slice streams from global memory through registers to its
//             shifted place; the new tuples go to delta at the tile's offset
//             and into the merged relation at co-rank + rank.
// No block waits on another.  Full and New are read once by the write pass
// and the merged Full and delta written once; the count pass adds New, the
// co-ranks, and the Full slices of dense tiles.
#include "kernels.h"

namespace cdl {

namespace {

constexpr int kDT = 256;
constexpr int kDItems = 16;
constexpr int kDTile = kDT * kDItems;  // merged items per tile
constexpr uint32_t kRepeat = 0xFFFFFFFFu;

template <int K>
__device__ __forceinline__ bool g_le(const ColsIn& a, uint64_t i, const ColsIn& b, uint64_t j) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t x = __ldg(a.c[k] + i), y = __ldg(b.c[k] + j);
    if (x != y) return x < y;
  }
  return true;
}

// Number of Full tuples among the first d of the merged order.
template <int K>
__device__ __forceinline__ uint64_t merge_split(const ColsIn& F, uint64_t nF, const ColsIn& U,
                                                uint64_t nU, uint64_t d) {
  uint64_t lo = d > nU ? d - nU : 0, hi = d < nF ? d : nF;
  while (lo < hi) {
    const uint64_t mid = lo + ((hi - lo) >> 1);
    if (g_le<K>(F, mid, U, d - mid - 1))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Inside a captured round, Full and the sizes come from device memory;
// false when the merged relation would not fit its buffer.
__device__ __forceinline__ bool resolve(const DevMerge& dm, ColsIn& F, uint64_t& nF, uint64_t& nU,
                                        uint64_t& ntiles) {
  if (!dm.n_full) return true;
  F = *dm.full;
  nF = dev_size(dm.n_full, nF);
  nU = dev_size(dm.n_fresh, nU);
  ntiles = (nF + nU + kDTile - 1) / kDTile;
  return nF + nU <= dm.cap_merged;
}

template <int K>
__global__ void k_merge_splits(ColsIn F, uint64_t nF, ColsIn U, uint64_t nU,
                               uint64_t* __restrict__ splits, uint64_t ntiles, DevMerge dm,
                               uint64_t* d_tiles) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool fits = resolve(dm, F, nF, nU, ntiles);
  if (d_tiles && t == 0) *d_tiles = fits ? ntiles : 0;  // the scan's length (0: nothing fits)
  if (!fits) {
    if (t == 0) atomicOr(dm.overflow, 1u);
    return;
  }
  if (t > ntiles) return;
  const uint64_t d = t * kDTile < nF + nU ? t * kDTile : nF + nU;
  splits[t] = merge_split<K>(F, nF, U, nU, d);
}

// Co-ranks (or kRepeat) of the New tuples j + 32 q, q < Q (those below b1),
// against the Full slice F[a0, a1) in global memory: the Q binary searches
// step together, so each step issues Q independent loads per column and
// their latencies overlap.  Every column of the probed Full tuple is read
// at once, and equality is noted on the way: the search for the count of
// tuples <= v tests the last one, so v is in the slice exactly when some
// tested tuple equals it.  The tuple before the slice (same for the whole
// tile) and the New tuple before j + 32 q are read up front.
template <int K, int Q>
__device__ __forceinline__ void co_ranks_global(const ColsIn& F, const ColsIn& U, uint64_t a0,
                                                uint64_t a1, uint64_t j, uint64_t b1,
                                                uint32_t (&p)[Q]) {
  uint32_t v[Q][K];
  bool rep[Q];
  uint32_t lo[Q], hi[Q];
  const uint32_t na = (uint32_t)(a1 - a0);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const uint64_t jq = j + 32u * q;
    const bool live = jq < b1;
#pragma unroll
    for (int k = 0; k < K; ++k) v[q][k] = live ? __ldg(U.c[k] + jq) : 0u;
    bool r = live && jq > 0, f = live && a0 > 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (live && jq > 0) r &= __ldg(U.c[k] + jq - 1) == v[q][k];
      if (live && a0 > 0) f &= __ldg(F.c[k] + a0 - 1) == v[q][k];
    }
    rep[q] = r || f;  // a repeat of the New tuple before it, or of the Full tuple before the slice
    lo[q] = 0;
    hi[q] = live ? na : 0u;
  }
  for (;;) {
    bool any = false;
    uint32_t x[Q][K];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint32_t mid = (lo[q] + hi[q]) >> 1;
#pragma unroll
      for (int k = 0; k < K; ++k) x[q][k] = lo[q] < hi[q] ? __ldg(F.c[k] + a0 + mid) : 0u;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (lo[q] >= hi[q]) continue;
      any = true;
      const uint32_t mid = (lo[q] + hi[q]) >> 1;
      bool le = true, eq = true;
#pragma unroll
      for (int k = K - 1; k >= 0; --k) {  // lexicographic, column 0 most significant
        if (x[q][k] != v[q][k]) {
          le = x[q][k] < v[q][k];
          eq = false;
        }
      }
      if (le) {
        lo[q] = mid + 1;
        rep[q] |= eq;
      } else {
        hi[q] = mid;
      }
    }
    if (!any) break;
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) p[q] = rep[q] ? kRepeat : lo[q];
}

// Shared-memory position of tile item i: one padding word per 32, so that
// threads walking from splits about kDItems apart mostly hit distinct banks.
__device__ __forceinline__ uint32_t spad(uint32_t i) { return i + (i >> 5); }
constexpr int kSRow = kDTile + kDTile / 32;  // words per column of a staged tile

// Co-rank (or kRepeat) of New tuple j against a dense tile's Full slice of
// na tuples staged in shared memory: a binary search, then the last Full
// tuple <= it (or the one before the slice) and the New tuple before it
// tell whether it repeats.
template <int K>
__device__ __forceinline__ uint32_t co_rank_smem(const ColsIn& F, const ColsIn& U,
                                                 const uint32_t* s, uint64_t a0, uint32_t na,
                                                 uint64_t j) {
  uint32_t v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = __ldg(U.c[k] + j);
  bool rep = j > 0;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (j > 0) rep &= __ldg(U.c[k] + j - 1) == v[k];
  uint32_t lo = 0, hi = na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    bool le = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t x = s[k * kSRow + spad(mid)];
      if (x != v[k]) {
        le = x < v[k];
        break;
      }
    }
    if (le)
      lo = mid + 1;
    else
      hi = mid;
  }
  bool eq = lo > 0 || a0 > 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (lo > 0)
      eq &= s[k * kSRow + spad(lo - 1)] == v[k];
    else if (a0 > 0)
      eq &= __ldg(F.c[k] + a0 - 1) == v[k];
  }
  return rep || eq ? kRepeat : lo;
}

// Persistent over groups of `group` tiles (1..8; grid = resident blocks).
// Warp w takes tile w of the group: a tile without New tuples costs one
// store, a sparse one (New < Full / 16) is searched by its warp alone with
// cached global loads; dense tiles are then taken by the whole block, which
// stages their slices in shared memory and merges them.  So a round whose few new tuples
// meet a large Full keeps every warp busy instead of one block per tile,
// while a small merge (fewer tiles than eight per resident block) keeps one
// tile per block.
template <int K>
__global__ void __launch_bounds__(kDT) k_count_new(ColsIn F, ColsIn U, uint64_t nF, uint64_t nU,
                                                   const uint64_t* __restrict__ splits,
                                                   uint32_t* __restrict__ corank,
                                                   uint32_t* __restrict__ tile_cnt,
                                                   uint64_t ntiles, DevMerge dm, uint32_t group) {
  extern __shared__ uint32_t s[];  // K x kSRow: the Full and New slices of a dense tile
  if (!resolve(dm, F, nF, nU, ntiles)) return;
  __shared__ uint32_t red[kDT / 32 + 1];
  constexpr int kW = kDT / 32;
  __shared__ uint32_t dense[kW];
  __shared__ uint32_t n_dense;
  const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
  for (uint64_t g = blockIdx.x; g * group < ntiles; g += gridDim.x) {
    if (threadIdx.x == 0) n_dense = 0;
    __syncthreads();
    const uint64_t tile = g * group + warp;
    if (warp < group && tile < ntiles) {
      const uint64_t d0 = tile * kDTile;
      const uint64_t d1 = d0 + kDTile < nF + nU ? d0 + kDTile : nF + nU;
      const uint64_t a0 = splits[tile], a1 = splits[tile + 1];
      const uint64_t b0 = d0 - a0, b1 = d1 - a1;
      const uint64_t na = a1 - a0, nb = b1 - b0;
      if (nb * 16 < na || nb == 0) {
        // searches stepped together per lane: two for pairs, one for wider tuples
        constexpr int kQ = K <= 2 ? 2 : 1;
        uint32_t cnt = 0;
        for (uint64_t j = b0 + lane; j < b1; j += 32 * kQ) {
          uint32_t p[kQ];
          co_ranks_global<K, kQ>(F, U, a0, a1, j, b1, p);
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            if (j + 32u * q >= b1) break;
            corank[j + 32u * q] = p[q];
            cnt += p[q] == kRepeat ? 0u : 1u;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) tile_cnt[tile] = cnt;
      } else if (lane == 0) {
        dense[atomicAdd(&n_dense, 1u)] = warp;
      }
    }
    __syncthreads();
    const uint32_t nd = n_dense;
    for (uint32_t q = 0; q < nd; ++q) {
      const uint64_t t = g * group + dense[q];
      const uint64_t d0 = t * kDTile;
      const uint64_t d1 = d0 + kDTile < nF + nU ? d0 + kDTile : nF + nU;
      const uint64_t a0 = splits[t], a1 = splits[t + 1];
      const uint64_t b0 = d0 - a0, b1 = d1 - a1;
      const uint32_t na = (uint32_t)(a1 - a0), nb = (uint32_t)(b1 - b0), nm = na + nb;
      // New at least a quarter of Full: both slices merged again; fewer New
      // tuples: each searches the staged Full slice
      const bool walk = (uint64_t)nb * 4 >= na;
      const uint32_t nst = walk ? nm : na;
      // stage the slices, eight loads per column in flight: Full at items
      // [0, na), New (walk only) at [na, nm) of each column's row of s
      constexpr int kS = 8;
      for (uint32_t base = 0; base < nst; base += kS * kDT) {
        uint32_t v[kS][K];
#pragma unroll
        for (int u = 0; u < kS; ++u) {
          const uint32_t i = base + u * kDT + threadIdx.x;
#pragma unroll
          for (int k = 0; k < K; ++k)
            v[u][k] = i < na ? __ldg(F.c[k] + a0 + i) : i < nm ? __ldg(U.c[k] + b0 + (i - na)) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kS; ++u) {
          const uint32_t i = base + u * kDT + threadIdx.x;
          if (i < nst) {
#pragma unroll
            for (int k = 0; k < K; ++k) s[k * kSRow + spad(i)] = v[u][k];
          }
        }
      }
      __syncthreads();
      // each thread merges kDItems items of the tile from its merge-path
      // split (Full before an equal New tuple): a New tuple's co-rank is the
      // number of Full tuples passed, and it repeats the last Full tuple
      // passed or the New tuple before it
      uint32_t cnt = 0;
      const uint32_t m0 = threadIdx.x * kDItems < nm ? threadIdx.x * kDItems : nm;
      const uint32_t m1 = m0 + kDItems < nm ? m0 + kDItems : nm;
      if (!walk) {
        for (uint64_t j = b0 + threadIdx.x; j < b1; j += kDT) {
          const uint32_t p = co_rank_smem<K>(F, U, s, a0, na, j);
          corank[j] = p;
          cnt += p == kRepeat ? 0u : 1u;
        }
      } else if (m0 < m1) {
        auto at = [&](uint32_t i, int k) { return s[k * kSRow + spad(i)]; };
        auto le_items = [&](uint32_t x, uint32_t y) {  // item x <= item y (s positions)
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const uint32_t a = at(x, k), b = at(y, k);
            if (a != b) return a < b;
          }
          return true;
        };
        uint32_t lo = m0 > nb ? m0 - nb : 0, hi = m0 < na ? m0 : na;
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          if (le_items(mid, na + (m0 - mid - 1)))
            lo = mid + 1;
          else
            hi = mid;
        }
        uint32_t i = lo, jn = m0 - lo;  // Full and New tuples before the thread's items
        uint32_t lf[K], ln[K];           // last Full and last New tuple passed
        bool hf = i > 0 || a0 > 0, hn = jn > 0 || b0 > 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          lf[k] = i > 0 ? at(i - 1, k) : a0 > 0 ? __ldg(F.c[k] + a0 - 1) : 0u;
          ln[k] = jn > 0 ? at(na + jn - 1, k) : b0 > 0 ? __ldg(U.c[k] + b0 - 1) : 0u;
        }
        for (uint32_t m = m0; m < m1; ++m) {
          bool take_full = jn >= nb;
          if (!take_full && i < na) take_full = le_items(i, na + jn);
          if (take_full) {
#pragma unroll
            for (int k = 0; k < K; ++k) lf[k] = at(i, k);
            hf = true;
            ++i;
          } else {
            uint32_t v[K];
            bool ef = hf, en = hn;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              v[k] = at(na + jn, k);
              ef &= lf[k] == v[k];
              en &= ln[k] == v[k];
            }
            const bool rep = ef || en;
            corank[b0 + jn] = rep ? kRepeat : i;
            cnt += rep ? 0u : 1u;
#pragma unroll
            for (int k = 0; k < K; ++k) ln[k] = v[k];
            hn = true;
            ++jn;
          }
        }
      }
      uint32_t tot;
      block_exclusive_sum<kDT, uint32_t>(cnt, red, &tot);
      if (threadIdx.x == 0) tile_cnt[t] = tot;
      __syncthreads();  // the next dense tile reuses s and red
    }
  }
}

// shift table index with one padding word per 32 (blocked scans stay
// free of bank conflicts)
__device__ __forceinline__ uint32_t pad(uint32_t i) { return i + (i >> 5); }
constexpr int kShiftWords = kDTile + 1 + (kDTile + 1) / 32 + 1;

template <int K>
__global__ void __launch_bounds__(kDT, 5) k_merge_write(ColsIn F, uint64_t nF, ColsIn U, uint64_t nU,
                                                     const uint64_t* __restrict__ splits,
                                                     const uint32_t* __restrict__ corank,
                                                     const uint64_t* __restrict__ tile_pre,
                                                     ColsOut D, ColsOut M, DevMerge dm,
                                                     uint64_t ntiles) {
  __shared__ uint32_t shift[kShiftWords];
  __shared__ uint32_t red[kDT / 32 + 1];
  if (!resolve(dm, F, nF, nU, ntiles)) return;  // (inside a captured round: sizes from the device)
  if (dm.n_full) {
    D = *dm.delta;
    M = *dm.merged;
  }
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  const uint64_t d0 = tile * kDTile;
  const uint64_t d1 = d0 + kDTile < nF + nU ? d0 + kDTile : nF + nU;
  const uint64_t a0 = splits[tile], a1 = splits[tile + 1];
  const uint64_t b0 = d0 - a0, b1 = d1 - a1;
  const uint32_t na = (uint32_t)(a1 - a0), nb = (uint32_t)(b1 - b0);
  const uint64_t dpre = tile_pre[tile];
  const uint64_t mbase = a0 + dpre;
  const bool merged = M.c[0] != nullptr;
  uint32_t tot_new = 0;
  if (nb) {
    // New tuples, blocked: thread owns [j0, j1) so that ranks follow order
    const uint32_t m = (nb + kDT - 1) / kDT;
    const uint32_t j0 = threadIdx.x * m < nb ? threadIdx.x * m : nb;
    const uint32_t j1 = j0 + m < nb ? j0 + m : nb;
    uint32_t p[kDItems];
    uint32_t newmask = 0;
#pragma unroll
    for (int q = 0; q < kDItems; ++q) {
      p[q] = kRepeat;
      if (j0 + q < j1) p[q] = __ldg(corank + b0 + j0 + q);
      if (p[q] != kRepeat) newmask |= 1u << q;
    }
    const uint32_t rank0 = block_exclusive_sum<kDT, uint32_t>(__popc(newmask), red, &tot_new);
    if (tot_new && merged) {
      for (uint32_t i = threadIdx.x; i <= na; i += kDT) shift[pad(i)] = 0;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kDItems; ++q)
        if ((newmask >> q) & 1u) atomicAdd(&shift[pad(p[q])], 1u);
      __syncthreads();
      const uint32_t c0 = threadIdx.x * kDItems;  // blocked inclusive scan over [0, na]
      uint32_t run = 0;
#pragma unroll
      for (int q = 0; q < kDItems; ++q) run += c0 + q <= na ? shift[pad(c0 + q)] : 0u;
      uint32_t tot;
      uint32_t acc = block_exclusive_sum<kDT, uint32_t>(run, red, &tot);
#pragma unroll
      for (int q = 0; q < kDItems; ++q)
        if (c0 + q <= na) {
          acc += shift[pad(c0 + q)];
          shift[pad(c0 + q)] = acc;
        }
    }
#pragma unroll
    for (int q = 0; q < kDItems; ++q) {
      if ((newmask >> q) & 1u) {
        const uint32_t r = rank0 + __popc(newmask & ((1u << q) - 1u));
        const uint64_t j = b0 + j0 + q;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const uint32_t v = __ldg(U.c[k] + j);
          D.c[k][dpre + r] = v;
          if (merged) M.c[k][mbase + p[q] + r] = v;
        }
      }
    }
    __syncthreads();
  }
  // the Full slice, four loads in flight per thread and column
  constexpr int kU = 8;
  for (uint32_t base = 0; merged && base < na; base += kU * kDT) {
    uint32_t v[kU][K];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t i = base + u * kDT + threadIdx.x;
#pragma unroll
      for (int k = 0; k < K; ++k) v[u][k] = i < na ? __ldg(F.c[k] + a0 + i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t i = base + u * kDT + threadIdx.x;
      if (i < na) {
        const uint64_t at = mbase + i + (tot_new ? shift[pad(i)] : 0u);
#pragma unroll
        for (int k = 0; k < K; ++k) M.c[k][at] = v[u][k];
      }
    }
  }
  __syncthreads();  // the next tile rebuilds the shift table
  }
}

uint64_t dm_tiles(uint64_t n_full, uint64_t n_fresh) {
  return (n_full + n_fresh + kDTile - 1) / kDTile;
}


size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

template <int K>
cudaError_t run_diff_merge(Ctx& c, ColsIn full, uint64_t n_full, ColsIn fresh, uint64_t n_fresh,
                           ColsOut delta, ColsOut merged, uint64_t* d_ndelta, void* ws,
                           const DevMerge& dm) {
  const uint64_t tiles = dm_tiles(n_full, n_fresh);
  char* w = static_cast<char*>(ws);
  uint64_t* splits = reinterpret_cast<uint64_t*>(w);
  w += up256((tiles + 1) * 8);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(w);
  w += up256(tiles * 4);
  uint64_t* pre = reinterpret_cast<uint64_t*>(w);
  w += up256(tiles * 8);
  uint32_t* corank = reinterpret_cast<uint32_t*>(w);
  w += up256((n_fresh ? n_fresh : 1) * 4);
  void* scan_ws = w;
  uint64_t* d_tiles = nullptr;  // device-sized: the scan's length (the split kernel writes it)
  if (dm.n_full) d_tiles = reinterpret_cast<uint64_t*>(w + scan_workspace(tiles));
  const size_t smem_count = sizeof(uint32_t) * K * kSRow;
  // blocks of k_count_new<K> a whole GPU holds at once, per device
  constexpr int kDevices = 64;
  static int resident_of[kDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int& resident = resident_of[dev < kDevices ? dev : 0];
  if (!resident) {
    e = cudaFuncSetAttribute(k_count_new<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_count);
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_new<K>, kDT, smem_count);
    if (e != cudaSuccess) return e;
    resident = (per_sm > 0 ? per_sm : 1) * sms;
  }
  // tiles per group: eight once there are eight per resident block, else
  // fewer, down to one per block for small merges
  uint64_t group = tiles / (uint64_t)resident;
  group = group < 1 ? 1 : (group > (uint64_t)(kDT / 32) ? (uint64_t)(kDT / 32) : group);
  const uint64_t groups = (tiles + group - 1) / group;
  const uint64_t count_grid = groups < (uint64_t)resident ? groups : (uint64_t)resident;
  {
    // New read, co-ranks written; Full sectors are read only where touched
    ProfScope p(c, kDiffCount, (4.0 * K + 4.0) * n_fresh);
    k_merge_splits<K><<<(unsigned)((tiles + 1 + 255) / 256), 256, 0, c.st>>>(
        full, n_full, fresh, n_fresh, splits, tiles, dm, d_tiles);
    k_count_new<K><<<(unsigned)count_grid, kDT, smem_count, c.st>>>(
        full, fresh, n_full, n_fresh, splits, corank, cnt, tiles, dm, (uint32_t)group);
  }
  {
    const int sc = c.scan_cls;  // the tile counts' scan is timed with the count pass
    c.scan_cls = kDiffCount;
    e = exclusive_scan(c, cnt, tiles, pre, d_ndelta, scan_ws, d_tiles);
    c.scan_cls = sc;
  }
  if (e != cudaSuccess) return e;
  // the step's algorithmic bytes: Full and New read, Full written again (the
  // co-ranks this pass also reads are the count pass's overhead); the delta
  // part of the writes (merged and delta) is added once its size is known
  const double mb = merged.c[0] ? 4.0 * K * n_full : 0.0;
  ProfScope p(c, kDiffMerge, 4.0 * K * (n_full + n_fresh) + mb);
  k_merge_write<K><<<dev_grid(tiles, dm.n_full), kDT, 0, c.st>>>(
      full, n_full, fresh, n_fresh, splits, corank, pre, delta, merged, dm, tiles);
  return cudaGetLastError();
}

}  // namespace

size_t diff_merge_workspace(uint64_t n_full, uint64_t n_fresh) {
  const uint64_t tiles = dm_tiles(n_full, n_fresh);
  return up256((tiles + 1) * 8) + up256(tiles * 4) + up256(tiles * 8) +
         up256((n_fresh ? n_fresh : 1) * 4) + scan_workspace(tiles) + 256;
}

cudaError_t diff_merge(Ctx& c, uint32_t k, ColsIn full, uint64_t n_full, ColsIn fresh,
                       uint64_t n_fresh, ColsOut delta, ColsOut merged, uint64_t* d_ndelta,
                       void* ws, const DevMerge* dm) {
  if (n_full + n_fresh == 0) return cudaMemsetAsync(d_ndelta, 0, sizeof(uint64_t), c.st);
  const DevMerge none{};
  const DevMerge& d = dm ? *dm : none;
  switch (k) {
    case 1: return run_diff_merge<1>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws, d);
    case 2: return run_diff_merge<2>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws, d);
    case 3: return run_diff_merge<3>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws, d);
    case 4: return run_diff_merge<4>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws, d);
    case 5: return run_diff_merge<5>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws, d);
    case 6: return run_diff_merge<6>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws, d);
    case 7: return run_diff_merge<7>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws, d);
    case 8: return run_diff_merge<8>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws, d);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cdl
