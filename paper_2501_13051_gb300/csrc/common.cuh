// Shared device helpers of the column-oriented Datalog kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cdl.h"

namespace cdl {

constexpr int kMaxK = CDL_MAX_ARITY;
constexpr uint32_t kEmpty = CDL_EMPTY_KEY;

// Column sets passed by value to kernels: column k of a relation is c[k].
struct ColsIn {
  const uint32_t* c[kMaxK];
};
struct ColsOut {
  uint32_t* c[kMaxK];
};

// Error bits a kernel may raise in the engine's device status word.
enum : uint32_t {
  kErrTimeout = 1u,   // a bounded wait ran out
  kErrCapacity = 2u,  // an output cursor passed its capacity
  kErrValue = 4u,     // the reserved value was seen in input
  kErrTable = 8u      // a hash table had no free slot
};

// 32-bit finaliser of MurmurHash3 (Austin Appleby, public domain): a
// bijective mixer, so distinct keys never collide before masking.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t k) {
  k ^= k >> 16;
  k *= 0x85ebca6bu;
  k ^= k >> 13;
  k *= 0xc2b2ae35u;
  k ^= k >> 16;
  return k;
}

__host__ __device__ __forceinline__ uint32_t hash_key(uint32_t k0, uint32_t k1) {
  return mix32(k0 ^ mix32(k1 + 0x9e3779b9u));
}

// Hash slot of the hybrid index: key (one or two words) -> (start, count) in
// the build side sorted by key.  An empty slot has k0 == k1 == 0xFFFFFFFF.
struct __align__(16) Slot {
  uint32_t k0, k1, start, count;
};

__device__ __forceinline__ Slot load_slot(const Slot* t, uint64_t i) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(t) + i);
  return Slot{v.x, v.y, v.z, v.w};
}

// Linear-probing lookup; returns count (0 if absent) and start.
__device__ __forceinline__ uint32_t probe_table(const Slot* t, uint64_t mask, uint32_t k0,
                                                uint32_t k1, uint32_t* start) {
  uint64_t i = hash_key(k0, k1) & mask;
  for (uint64_t step = 0; step <= mask; ++step) {
    const Slot s = load_slot(t, i);
    if (s.k0 == k0 && s.k1 == k1) {
      *start = s.start;
      return s.count;
    }
    if (s.k0 == kEmpty && s.k1 == kEmpty) break;
    i = (i + 1) & mask;
  }
  *start = 0;
  return 0;
}

// Lexicographic comparison of tuples held in registers.
template <int K>
__device__ __forceinline__ bool tuple_le(const uint32_t (&a)[K], const uint32_t (&b)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (a[k] != b[k]) return a[k] < b[k];
  }
  return true;
}
template <int K>
__device__ __forceinline__ bool tuple_eq(const uint32_t (&a)[K], const uint32_t (&b)[K]) {
  bool e = true;
#pragma unroll
  for (int k = 0; k < K; ++k) e &= a[k] == b[k];
  return e;
}
template <int K>
__device__ __forceinline__ void load_tuple(const ColsIn& c, uint64_t i, uint32_t (&t)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) t[k] = c.c[k][i];
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Block-wide exclusive sum over THREADS threads (values per thread), with
// the block total in *total.  smem: THREADS/32 words.
template <int THREADS, typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* smem, T* total) {
  constexpr int W = THREADS / 32;
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= (uint32_t)o) inc += n;
  }
  if (lane == 31) smem[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < (uint32_t)W ? smem[lane] : T(0);
    T winc = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T n = __shfl_up_sync(0xffffffffu, winc, o);
      if (lane >= (uint32_t)o) winc += n;
    }
    if (lane < (uint32_t)W) smem[lane] = winc - w;
    if (lane == W - 1) smem[W] = winc;
  }
  __syncthreads();
  const T res = smem[warp] + inc - v;
  *total = smem[W];
  __syncthreads();
  return res;
}

// Exclusive max-scan over the block's threads (0 for thread 0).  smem:
// THREADS/32 words.  Ends with a barrier.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_max(uint32_t v, uint32_t* smem) {
  static_assert(THREADS % 32 == 0 && THREADS <= 1024, "whole warps");
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= (uint32_t)o) inc = n > inc ? n : inc;
  }
  const uint32_t ex_in_warp = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 31) smem[warp] = inc;
  __syncthreads();
  uint32_t before = 0;  // max over the earlier warps
  for (uint32_t w = 0; w < warp; ++w) before = smem[w] > before ? smem[w] : before;
  __syncthreads();
  const uint32_t own = lane > 0 ? ex_in_warp : 0u;
  return own > before ? own : before;
}

// A relation of arity k whose columns need T = bits_0 + ... + bits_{k-1}
// bits in all can also be held as a bitmap of 2^T bits: tuple (v_0..v_{k-1})
// is bit sum_k v_k << shift_k, with shift_k the bits of the columns after k.
// Increasing bit order is then the tuples' lexicographic order, and setting
// a bit twice is a no-op, so the bitmap is a sorted set.
struct DenseSet {
  uint32_t* words;  // nbits / 32 words (at least one)
  uint64_t nbits;   // 2^T
  uint32_t k;
  uint32_t shift[kMaxK];
  uint32_t mask[kMaxK];  // 2^bits_k - 1
};

// The word and bit of tuple v in d; false when v lies outside d.
__device__ __forceinline__ bool dense_locate(const DenseSet& d, const uint32_t (&v)[kMaxK],
                                             uint32_t* word, uint32_t* bit) {
  uint64_t idx = 0;
  bool out = false;
#pragma unroll
  for (int k = 0; k < kMaxK; ++k)
    if (k < (int)d.k) {
      idx |= (uint64_t)v[k] << d.shift[k];
      out |= v[k] > d.mask[k];
    }
  *word = (uint32_t)(idx >> 5);
  *bit = 1u << (idx & 31);
  return !out && idx < d.nbits;
}

// Bits only go from 0 to 1 while tuples are added, so a bit seen set (in a
// value read at any time, from L1 or L2) is set: only a missing bit needs an
// atomic.  Repeated outputs of a join mostly stop at the read.  (Merging a
// warp's bits per word first, by match and reduce, costs more than it
// saves: those warp instructions then bound the join's write pass.)
__device__ __forceinline__ bool dense_missing(const DenseSet& d, uint32_t word, uint32_t bit) {
  return (d.words[word] & bit) == 0u;
}

// Sets the bit of tuple v (keep = the thread has one); a tuple outside the
// bitmap raises kErrCapacity and sets nothing.
__device__ __forceinline__ void dense_set_bits(const DenseSet& d, const uint32_t (&v)[kMaxK],
                                               bool keep, uint32_t* err) {
  uint32_t word = 0, bit = 0;
  if (!keep) return;
  if (!dense_locate(d, v, &word, &bit)) {
    atomicOr(err, kErrCapacity);
    return;
  }
  if (dense_missing(d, word, bit)) atomicOr(d.words + word, bit);
}

// Device-sized launches (a round captured in a CUDA graph): the grid is
// sized for a capacity known to the host, the actual size is read from
// device memory and clamped to that capacity, so no access can leave the
// buffers the capacity describes.  dn == nullptr: the size is `cap` itself.
__device__ __forceinline__ uint64_t dev_size(const uint64_t* dn, uint64_t cap) {
  if (!dn) return cap;
  const uint64_t v = *dn;
  return v < cap ? v : cap;
}

// Grid of a launch over `tiles` tiles.  A device-sized launch (dn set: a
// captured round, its tiles counted for a capacity) gets at most kDevGrid
// blocks, which loop over the tiles the actual size gives, so that rounds
// far below the capacity do not launch blocks by the hundred thousand;
// other launches get one block per tile (one iteration of the loop).
constexpr uint64_t kDevGrid = 152 * 8;
inline unsigned dev_grid(uint64_t tiles, const void* dn) {
  return (unsigned)(dn && tiles > kDevGrid ? kDevGrid : (tiles ? tiles : 1));
}

}  // namespace cdl
