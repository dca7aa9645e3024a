// Step (a): the hybrid index of Section 3.  Over a column (or column pair)
// sorted by value, every distinct key gets one open-addressing slot holding
// (key, start, count): the first position of the key in the sorted order and
// its run length (the run-length encoding the paper stores in its "unique
// hashmap").  Linear probing over a power-of-two table; the hash is the
// MurmurHash3 finaliser.
//
// One pass: the thread at a run head finds the end of its run by galloping
// (exponential then binary search over the sorted keys, O(log run) reads,
// so a hot key with a long run costs one thread a few dozen reads rather
// than a walk), then claims a slot with a 64-bit compare-and-swap on the
// key words.  Keys are distinct, so an insert never meets its own key.
#include "kernels.h"

namespace cdl {

namespace {

constexpr int kThreads = 256;
constexpr unsigned long long kEmpty64 = ~0ull;

template <bool TWO>
__device__ __forceinline__ bool key_ne(const uint32_t* k0, const uint32_t* k1, uint64_t i,
                                       uint32_t a0, uint32_t a1) {
  if (TWO) return __ldg(k0 + i) != a0 || __ldg(k1 + i) != a1;
  return __ldg(k0 + i) != a0;
}

template <bool TWO>
__global__ void __launch_bounds__(kThreads) k_hash_build(const uint32_t* __restrict__ k0,
                                                         const uint32_t* __restrict__ k1,
                                                         uint64_t n, Slot* __restrict__ t,
                                                         uint64_t mask, uint32_t* err) {
  const uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  const uint32_t a0 = __ldg(k0 + i);
  const uint32_t a1 = TWO ? __ldg(k1 + i) : 0u;
  if (i > 0 && !key_ne<TWO>(k0, k1, i - 1, a0, a1)) return;  // not a run head
  // gallop to the first position past the run
  uint64_t lo = i + 1, hi = n, step = 1;
  while (true) {
    const uint64_t j = i + step;
    if (j >= n) break;
    if (key_ne<TWO>(k0, k1, j, a0, a1)) {
      hi = j;
      break;
    }
    lo = j + 1;
    step <<= 1;
  }
  while (lo < hi) {
    const uint64_t mid = lo + ((hi - lo) >> 1);
    if (key_ne<TWO>(k0, k1, mid, a0, a1))
      hi = mid;
    else
      lo = mid + 1;
  }
  const uint64_t end = lo;
  const unsigned long long packed = ((unsigned long long)a1 << 32) | a0;
  uint64_t s = hash_key(a0, a1) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const unsigned long long prev =
        atomicCAS(reinterpret_cast<unsigned long long*>(t + s), kEmpty64, packed);
    if (prev == kEmpty64) {
      t[s].start = (uint32_t)i;
      t[s].count = (uint32_t)(end - i);
      return;
    }
    s = (s + 1) & mask;
  }
  if (err) atomicOr(err, kErrTable);
}

template <bool TWO>
__global__ void __launch_bounds__(kThreads) k_count_heads(const uint32_t* __restrict__ k0,
                                                          const uint32_t* __restrict__ k1,
                                                          uint64_t n, unsigned long long* out) {
  uint32_t mine = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * kThreads) {
    const uint32_t a0 = __ldg(k0 + i), a1 = TWO ? __ldg(k1 + i) : 0u;
    mine += (i == 0 || key_ne<TWO>(k0, k1, i - 1, a0, a1)) ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if (lane_id() == 0 && mine) atomicAdd(out, (unsigned long long)mine);
}

}  // namespace

uint64_t table_slots(uint64_t n_keys, double load) {
  if (load <= 0.0 || load > 0.9) load = 0.5;
  uint64_t want = (uint64_t)((double)(n_keys ? n_keys : 1) / load) + 1;
  uint64_t s = 16;
  while (s < want) s <<= 1;
  return s;
}

cudaError_t hash_build(Ctx& c, const uint32_t* k0, const uint32_t* k1, uint64_t n, Slot* table,
                       uint64_t slots) {
  cudaError_t e = cudaMemsetAsync(table, 0xFF, slots * sizeof(Slot), c.st);
  if (e != cudaSuccess || n == 0) return e;
  ProfScope p(c, kHashBuild, (k1 ? 8.0 : 4.0) * n);
  const unsigned grid = (unsigned)((n + kThreads - 1) / kThreads);
  if (k1)
    k_hash_build<true><<<grid, kThreads, 0, c.st>>>(k0, k1, n, table, slots - 1, c.d_err);
  else
    k_hash_build<false><<<grid, kThreads, 0, c.st>>>(k0, k1, n, table, slots - 1, c.d_err);
  return cudaGetLastError();
}

cudaError_t count_heads(Ctx& c, const uint32_t* k0, const uint32_t* k1, uint64_t n,
                        uint64_t* d_out) {
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(uint64_t), c.st);
  if (e != cudaSuccess || n == 0) return e;
  ProfScope p(c, kCountHeads, (k1 ? 8.0 : 4.0) * n);
  uint64_t blocks = (n + kThreads * 8 - 1) / (kThreads * 8);
  if (blocks > 152 * 16) blocks = 152 * 16;
  auto* out = reinterpret_cast<unsigned long long*>(d_out);
  if (k1)
    k_count_heads<true><<<(unsigned)blocks, kThreads, 0, c.st>>>(k0, k1, n, out);
  else
    k_count_heads<false><<<(unsigned)blocks, kThreads, 0, c.st>>>(k0, k1, n, out);
  return cudaGetLastError();
}

}  // namespace cdl
