// Selection / projection of one body atom (Section 4, "Projection and
// Selection"): rows are filtered on constants, repeated variables and
// inequalities, then projected onto head columns and packed with one atomic
// per block; plus the check of loaded values against the reserved value.
#include "kernels.h"

namespace cdl {

namespace {

// ------------------------------------------------------------- select
constexpr int kST = 256;
constexpr int kSItems = 8;

__device__ __forceinline__ uint32_t sel_ref(const SelectSpec& s, const Ref& r, uint64_t row) {
  return r.side == 2 ? r.v : __ldg(s.in.c[r.v] + row);
}

__global__ void __launch_bounds__(kST) k_select(const SelectSpec s, ColsOut out,
                                                unsigned long long* cursor, uint64_t cap,
                                                uint32_t* err) {
  __shared__ uint32_t red[kST / 32 + 1];
  __shared__ unsigned long long s_base;
  const uint64_t base = (uint64_t)blockIdx.x * kST * kSItems;
  for (int it = 0; it < kSItems; ++it) {
    const uint64_t row = base + (uint64_t)it * kST + threadIdx.x;
    bool keep = row < s.n;
    uint32_t vals[kMaxK] = {0, 0, 0, 0};
    if (keep) {
      for (uint32_t q = 0; q < s.n_const; ++q)
        keep &= __ldg(s.in.c[s.const_col[q]] + row) == s.const_val[q];
      for (uint32_t q = 0; q < s.n_same; ++q)
        keep &= __ldg(s.in.c[s.same[q][0]] + row) == __ldg(s.in.c[s.same[q][1]] + row);
      for (uint32_t q = 0; q < s.n_neq; ++q)
        keep &= sel_ref(s, s.neq[q][0], row) != sel_ref(s, s.neq[q][1], row);
#pragma unroll
      for (int k = 0; k < kMaxK; ++k)
        if (k < (int)s.out_k) vals[k] = sel_ref(s, s.out[k], row);
    }
    uint32_t cnt;
    const uint32_t local = block_exclusive_sum<kST, uint32_t>(keep ? 1u : 0u, red, &cnt);
    if (threadIdx.x == 0) s_base = cnt ? atomicAdd(cursor, (unsigned long long)cnt) : 0ull;
    __syncthreads();
    const uint64_t pos = s_base + local;
    __syncthreads();
    if (keep) {
      if (pos < cap) {
#pragma unroll
        for (int k = 0; k < kMaxK; ++k)
          if (k < (int)s.out_k) out.c[k][pos] = vals[k];
      } else {
        if (err) atomicOr(err, kErrCapacity);
      }
    }
  }
}

__global__ void k_check_values(ColsIn in, uint32_t k, uint64_t n, uint32_t* d_max,
                               uint32_t* err) {
  for (uint32_t c = 0; c < k; ++c) {
    uint32_t m = 0;
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
      const uint32_t v = __ldg(in.c[c] + i);
      bad |= v == kEmpty;
      m = max(m, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (bad && err) atomicOr(err, kErrValue);
    if (lane_id() == 0) atomicMax(d_max + c, m);
  }
}

// Batched fixpoints: the delta of a relation whose column 0 is an instance
// id is sorted by instance, so every run head marks an instance that derived
// something in this round.
__global__ void k_mark_instances(const uint32_t* __restrict__ inst, uint64_t n,
                                 uint32_t n_instances, uint64_t* __restrict__ last_round,
                                 uint64_t round, const ColsIn* dinst, const uint64_t* dn,
                                 const uint64_t* dround) {
  if (dinst) {  // inside a captured round: the delta and the round from device memory
    inst = dinst->c[0];
    n = dev_size(dn, n);
    round += *dround;
  }
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = __ldg(inst + i);
    if ((i == 0 || __ldg(inst + i - 1) != v) && v < n_instances) last_round[v] = round;
  }
}

// bounds[i] = the first row whose instance id (column 0, sorted) is >= i,
// for i in [0, n_instances].
__global__ void k_instance_bounds(const uint32_t* __restrict__ inst, uint64_t n,
                                  uint32_t n_instances, uint64_t* __restrict__ bounds) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n_instances) return;
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if ((uint64_t)__ldg(inst + mid) < i)
      lo = mid + 1;
    else
      hi = mid;
  }
  bounds[i] = lo;
}

// Output row j of segment s (out_off[s] <= j < out_off[s + 1]) copies row
// src[s] + (j - out_off[s]) of table a, or of table b when bit 63 of src[s]
// is set.  Consecutive rows of a segment are consecutive source rows, so
// reads and writes stay coalesced.
constexpr int kGT = 256;
constexpr int kGItems = 8;
constexpr uint32_t kGSmem = 2048;  // segment offsets held in shared memory

template <bool SMEM>
__global__ void __launch_bounds__(kGT) k_gather_segments(ColsIn a, ColsIn b, uint32_t k,
                                                         const uint64_t* __restrict__ out_off,
                                                         const uint64_t* __restrict__ src,
                                                         uint32_t nseg, uint64_t total,
                                                         ColsOut out) {
  __shared__ uint64_t s_off[SMEM ? kGSmem + 1 : 1];
  if (SMEM) {
    for (uint32_t i = threadIdx.x; i <= nseg; i += kGT) s_off[i] = out_off[i];
    __syncthreads();
  }
  const uint64_t base = (uint64_t)blockIdx.x * kGT * kGItems;
  for (int it = 0; it < kGItems; ++it) {
    const uint64_t j = base + (uint64_t)it * kGT + threadIdx.x;
    if (j >= total) break;
    uint32_t lo = 0, hi = nseg;  // the last segment whose start is <= j
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      const uint64_t o = SMEM ? s_off[mid] : __ldg(out_off + mid);
      if (o <= j)
        lo = mid;
      else
        hi = mid;
    }
    const uint64_t start = SMEM ? s_off[lo] : __ldg(out_off + lo);
    const uint64_t sv = __ldg(src + lo);
    const uint64_t row = (sv & ~(1ull << 63)) + (j - start);
    const bool from_b = (sv >> 63) != 0;
#pragma unroll
    for (int c = 0; c < kMaxK; ++c)  // constant indices: the column sets stay in registers
      if (c < (int)k) out.c[c][j] = __ldg((from_b ? b.c[c] : a.c[c]) + row);
  }
}

}  // namespace

// col[j] = s for every row j of segment s (rows [off[s], off[s + 1])).
__global__ void k_fill_segments(uint32_t* __restrict__ col, const uint64_t* __restrict__ off,
                                uint32_t nseg, uint64_t total) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total;
       j += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = nseg;  // the last segment starting at or before j
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(off + mid) <= j)
        lo = mid;
      else
        hi = mid;
    }
    col[j] = lo;
  }
}

cudaError_t fill_segments(Ctx& c, uint32_t* col, const uint64_t* off, uint32_t nseg,
                          uint64_t total) {
  if (total == 0 || nseg == 0) return cudaSuccess;
  ProfScope p(c, kMisc, 4.0 * total);
  uint64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_fill_segments<<<(unsigned)blocks, 256, 0, c.st>>>(col, off, nseg, total);
  return cudaGetLastError();
}

// Row j of segment s (rows [off[s], off[s + 1])): out.c[0][j] = s and
// out.c[1 + c][j] = column c of src[s] at row j - off[s].
__global__ void k_concat_segments(ColsOut out, const ColsIn* __restrict__ src, uint32_t k,
                                  const uint64_t* __restrict__ off, uint32_t nseg,
                                  uint64_t total) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total;
       j += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = nseg;  // the last segment starting at or before j
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(off + mid) <= j)
        lo = mid;
      else
        hi = mid;
    }
    const uint64_t r = j - __ldg(off + lo);
    out.c[0][j] = lo;
#pragma unroll
    for (uint32_t c = 0; c + 1 < (uint32_t)kMaxK; ++c)
      if (c < k) out.c[c + 1][j] = __ldg(src[lo].c[c] + r);
  }
}

cudaError_t concat_segments(Ctx& c, ColsOut out, const ColsIn* src, uint32_t k,
                            const uint64_t* off, uint32_t nseg, uint64_t total) {
  if (total == 0 || nseg == 0) return cudaSuccess;
  ProfScope p(c, kMisc, (8.0 * k + 4.0) * total);
  uint64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_concat_segments<<<(unsigned)blocks, 256, 0, c.st>>>(out, src, k, off, nseg, total);
  return cudaGetLastError();
}

cudaError_t instance_bounds(Ctx& c, const uint32_t* inst, uint64_t n, uint32_t n_instances,
                            uint64_t* bounds) {
  ProfScope p(c, kRetire, 8.0 * (n_instances + 1));
  k_instance_bounds<<<(n_instances + 256) / 256, 256, 0, c.st>>>(inst, n, n_instances, bounds);
  return cudaGetLastError();
}

cudaError_t gather_segments(Ctx& c, uint32_t k, ColsIn a, ColsIn b, const uint64_t* out_off,
                            const uint64_t* src, uint32_t nseg, uint64_t total, ColsOut out) {
  if (total == 0 || nseg == 0) return cudaSuccess;
  ProfScope p(c, kRetire, 8.0 * k * total);
  const uint64_t blocks = (total + kGT * kGItems - 1) / (kGT * kGItems);
  if (nseg <= kGSmem)
    k_gather_segments<true><<<(unsigned)blocks, kGT, 0, c.st>>>(a, b, k, out_off, src, nseg, total,
                                                                 out);
  else
    k_gather_segments<false><<<(unsigned)blocks, kGT, 0, c.st>>>(a, b, k, out_off, src, nseg,
                                                                  total, out);
  return cudaGetLastError();
}

cudaError_t mark_instances(Ctx& c, const uint32_t* inst, uint64_t n, uint32_t n_instances,
                           uint64_t* last_round, uint64_t round, const ColsIn* dinst,
                           const uint64_t* dn, const uint64_t* dround) {
  if (n == 0) return cudaSuccess;
  ProfScope p(c, kMisc, 4.0 * n);
  k_mark_instances<<<dev_grid((n + 255) / 256, dinst), 256, 0, c.st>>>(
      inst, n, n_instances, last_round, round, dinst, dn, dround);
  return cudaGetLastError();
}

cudaError_t select_project(Ctx& c, const SelectSpec& s, ColsOut out, uint64_t* d_cursor,
                           uint64_t out_cap, uint32_t* soft_overflow) {
  if (s.n == 0) return cudaSuccess;
  const uint64_t blocks = (s.n + kST * kSItems - 1) / (kST * kSItems);
  ProfScope p(c, kSelect, 4.0 * s.in_k * s.n + 4.0 * s.out_k * s.n);
  k_select<<<(unsigned)blocks, kST, 0, c.st>>>(s, out,
                                               reinterpret_cast<unsigned long long*>(d_cursor),
                                               out_cap,
                                               soft_overflow ? soft_overflow : c.d_err);
  return cudaGetLastError();
}

cudaError_t check_values(Ctx& c, ColsIn in, uint32_t k, uint64_t n, uint32_t* d_max) {
  cudaError_t e = cudaMemsetAsync(d_max, 0, sizeof(uint32_t) * k, c.st);
  if (e != cudaSuccess || n == 0) return e;
  ProfScope p(c, kMisc, 4.0 * k * n);
  uint64_t blocks = (n + 2047) / 2048;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_check_values<<<(unsigned)blocks, 256, 0, c.st>>>(in, k, n, d_max, c.d_err);
  return cudaGetLastError();
}

}  // namespace cdl
