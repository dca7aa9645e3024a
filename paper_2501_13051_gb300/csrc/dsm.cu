// Algorithm 2: deduplication of new tuples against Full in the decomposed
// storage model (Section 3, "Column-Oriented Relations on the GPU"; Section
// 4, "Union and Deduplication").  Full keeps its rows in insertion order,
// the row number being the tuple's surrogate id, and every column k has
//   * a sorted index: the ids in order of (value, id), stored beside the
//     values themselves (ids ascend within one value), and
//   * the unique hashmap over that order: value -> (start, count) of its run.
// A new tuple t belongs to Full exactly when the id ranges of its values,
// one per column, share an id (the paper's "overlap" of the ranges; the
// join New |x| Reach_0 |x|_{id,y} Reach_1 of Section 4).  A tuple whose
// value is missing from some column's hashmap is new at once (Algorithm 2
// drops empty ranges before the overlap test).  The test walks the smallest
// of the ranges and compares each id's values in the other columns with t.
//
// The ablation the paper argues against (Section 3: repeated values make a
// plain hashmap's probe chains long) is the hash-only index: one
// open-addressing multimap of (value, id) entries, one per row of column 0,
// probed by walking the chain of t's first value.
//
// New rows arrive sorted (step c); a row equal to the row before it is a
// repeat.  A flag per row (1 = new) is scanned and the new rows compacted,
// so delta comes out sorted.
#include "kernels.h"

namespace cdl {

namespace {

constexpr int kPT = 256;
constexpr unsigned long long kMmEmpty = ~0ull;

template <int K, bool HASH_ONLY>
__global__ void __launch_bounds__(kPT) k_dsm_probe(ColsIn rows, uint64_t n, DsmView v,
                                                   uint32_t* __restrict__ flags, uint32_t* err) {
  const uint64_t i = (uint64_t)blockIdx.x * kPT + threadIdx.x;
  if (i >= n) return;
  uint32_t t[K];
#pragma unroll
  for (int k = 0; k < K; ++k) t[k] = __ldg(rows.c[k] + i);
  bool rep = i > 0;
  if (i > 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) rep &= __ldg(rows.c[k] + i - 1) == t[k];
  }
  bool member = false;
  if (!rep && v.n) {
    if (HASH_ONLY) {
      uint64_t s = hash_key(t[0], 0u) & v.mm_mask;
      const unsigned long long* mm = reinterpret_cast<const unsigned long long*>(v.mm);
      for (uint64_t probe = 0; probe <= v.mm_mask && !member; ++probe) {
        const unsigned long long e = mm[s];
        if (e == kMmEmpty) break;
        if ((uint32_t)e == t[0]) {
          const uint32_t id = (uint32_t)(e >> 32);
          bool eq = true;
#pragma unroll
          for (int k = 1; k < K; ++k) eq &= __ldg(v.raw.c[k] + id) == t[k];
          member = eq;
        }
        s = (s + 1) & v.mm_mask;
      }
    } else {
      uint32_t start[K], cnt[K];
      bool empty = false;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        cnt[k] = probe_table(v.table[k], v.mask[k], t[k], 0u, &start[k]);
        empty |= cnt[k] == 0;
      }
      if (!empty) {
        int km = 0;
#pragma unroll
        for (int k = 1; k < K; ++k)
          if (cnt[k] < cnt[km]) km = k;
        const uint32_t* ids = v.ids[km];
        const uint32_t s0 = start[km], s1 = start[km] + cnt[km];
        for (uint32_t j = s0; j < s1 && !member; ++j) {
          const uint32_t id = __ldg(ids + j);
          bool eq = true;
#pragma unroll
          for (int k = 0; k < K; ++k)
            if (k != km) eq &= __ldg(v.raw.c[k] + id) == t[k];
          member = eq;
        }
      }
    }
  }
  flags[i] = (!rep && !member) ? 1u : 0u;
}

template <int K>
__global__ void __launch_bounds__(kPT) k_compact_rows(ColsIn rows, uint64_t n,
                                                      const uint32_t* __restrict__ flags,
                                                      const uint64_t* __restrict__ off,
                                                      ColsOut out) {
  const uint64_t i = (uint64_t)blockIdx.x * kPT + threadIdx.x;
  if (i >= n || !flags[i]) return;
  const uint64_t o = off[i];
#pragma unroll
  for (int k = 0; k < K; ++k) out.c[k][o] = __ldg(rows.c[k] + i);
}

__global__ void __launch_bounds__(kPT) k_mm_insert(const uint32_t* __restrict__ keys, uint64_t n,
                                                   uint32_t id0, unsigned long long* table,
                                                   uint64_t mask, uint32_t* err) {
  const uint64_t i = (uint64_t)blockIdx.x * kPT + threadIdx.x;
  if (i >= n) return;
  const uint32_t key = __ldg(keys + i);
  const unsigned long long e = ((unsigned long long)(id0 + (uint32_t)i) << 32) | key;
  uint64_t s = hash_key(key, 0u) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    if (atomicCAS(table + s, kMmEmpty, e) == kMmEmpty) return;
    s = (s + 1) & mask;
  }
  if (err) atomicOr(err, kErrTable);
}

__global__ void k_iota(uint32_t* __restrict__ out, uint64_t n, uint32_t first) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = first + (uint32_t)i;
}

template <int K>
cudaError_t launch_probe(Ctx& c, ColsIn rows, uint64_t n, const DsmView& v, bool hash_only,
                         uint32_t* flags) {
  const unsigned grid = (unsigned)((n + kPT - 1) / kPT);
  if (hash_only)
    k_dsm_probe<K, true><<<grid, kPT, 0, c.st>>>(rows, n, v, flags, c.d_err);
  else
    k_dsm_probe<K, false><<<grid, kPT, 0, c.st>>>(rows, n, v, flags, c.d_err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t dsm_probe(Ctx& c, uint32_t k, ColsIn rows, uint64_t n, const DsmView& v,
                      bool hash_only, uint32_t* flags) {
  if (n == 0) return cudaSuccess;
  // the rows read; the range walk's reads depend on the data
  ProfScope p(c, kDedup, 4.0 * k * n + 4.0 * n);
  switch (k) {
    case 1: return launch_probe<1>(c, rows, n, v, hash_only, flags);
    case 2: return launch_probe<2>(c, rows, n, v, hash_only, flags);
    case 3: return launch_probe<3>(c, rows, n, v, hash_only, flags);
    case 4: return launch_probe<4>(c, rows, n, v, hash_only, flags);
    case 5: return launch_probe<5>(c, rows, n, v, hash_only, flags);
    case 6: return launch_probe<6>(c, rows, n, v, hash_only, flags);
    case 7: return launch_probe<7>(c, rows, n, v, hash_only, flags);
    case 8: return launch_probe<8>(c, rows, n, v, hash_only, flags);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t compact_rows(Ctx& c, uint32_t k, ColsIn rows, uint64_t n, const uint32_t* flags,
                         const uint64_t* off, ColsOut out) {
  if (n == 0) return cudaSuccess;
  ProfScope p(c, kDedup, 4.0 * n + 8.0 * n);  // flags and offsets; the rows once known
  const unsigned grid = (unsigned)((n + kPT - 1) / kPT);
  switch (k) {
    case 1: k_compact_rows<1><<<grid, kPT, 0, c.st>>>(rows, n, flags, off, out); break;
    case 2: k_compact_rows<2><<<grid, kPT, 0, c.st>>>(rows, n, flags, off, out); break;
    case 3: k_compact_rows<3><<<grid, kPT, 0, c.st>>>(rows, n, flags, off, out); break;
    case 4: k_compact_rows<4><<<grid, kPT, 0, c.st>>>(rows, n, flags, off, out); break;
    case 5: k_compact_rows<5><<<grid, kPT, 0, c.st>>>(rows, n, flags, off, out); break;
    case 6: k_compact_rows<6><<<grid, kPT, 0, c.st>>>(rows, n, flags, off, out); break;
    case 7: k_compact_rows<7><<<grid, kPT, 0, c.st>>>(rows, n, flags, off, out); break;
    case 8: k_compact_rows<8><<<grid, kPT, 0, c.st>>>(rows, n, flags, off, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t mm_insert(Ctx& c, const uint32_t* keys, uint64_t n, uint32_t id0, uint2* table,
                      uint64_t slots) {
  if (n == 0) return cudaSuccess;
  ProfScope p(c, kDedup, 4.0 * n + 8.0 * n);
  k_mm_insert<<<(unsigned)((n + kPT - 1) / kPT), kPT, 0, c.st>>>(
      keys, n, id0, reinterpret_cast<unsigned long long*>(table), slots - 1, c.d_err);
  return cudaGetLastError();
}

cudaError_t iota_u32(Ctx& c, uint32_t* out, uint64_t n, uint32_t first) {
  if (n == 0) return cudaSuccess;
  k_iota<<<(unsigned)((n + 255) / 256), 256, 0, c.st>>>(out, n, first);
  return cudaGetLastError();
}

}  // namespace cdl
