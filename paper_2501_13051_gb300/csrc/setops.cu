// Step (d) and the per-atom copy step.
//
// Difference + merge (Section 4, "Union and Deduplication": delta = New -
// Full with the difference operator; Section 3, "Continuous Memory Layout":
// delta is merged eagerly into one contiguous sorted Full).  Both inputs are
// sorted; Full is unique, New may repeat.  The merged order takes a Full
// tuple before an equal New tuple, so a New tuple is a repeat exactly when it
// equals the Full tuple or the New tuple just before it in that order -- the
// removal of repeats (step c's "unique") is folded into this pass.  Tiles
// are merge-path splits of the combined sequence (Green, McColl & Bader,
// "GPU merge path", ICS 2012), loaded into shared memory; pass 1 counts
// each tile's new tuples, a scan turns the counts into delta offsets, pass 2
// writes delta and the merged relation (a tile's merged output starts at
// (Full tuples before the tile) + (new tuples before the tile)).
//
// Selection / projection (Section 4, "Projection and Selection") of one
// body atom: rows are filtered on constants, repeated variables and
// inequalities, then projected onto head columns, packed with one atomic
// per block and warp.
#include "kernels.h"

namespace cdl {

namespace {

constexpr int kMT = 256;
constexpr int kMItems = 8;
constexpr int kMTile = kMT * kMItems;

template <int K>
__device__ __forceinline__ bool g_le(const ColsIn& a, uint64_t i, const ColsIn& b, uint64_t j) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t x = __ldg(a.c[k] + i), y = __ldg(b.c[k] + j);
    if (x != y) return x < y;
  }
  return true;
}

// shared tile: column k of item i at s[k * kMTile + i]
template <int K>
__device__ __forceinline__ bool s_le(const uint32_t* s, uint32_t i, uint32_t j) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t x = s[k * kMTile + i], y = s[k * kMTile + j];
    if (x != y) return x < y;
  }
  return true;
}

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

template <int K, bool WRITE>
__global__ void __launch_bounds__(kMT) k_diff_merge(ColsIn F, uint64_t nF, ColsIn U, uint64_t nU,
                                                    uint32_t* __restrict__ cnt_out,
                                                    const uint64_t* __restrict__ pre, ColsOut D,
                                                    ColsOut M) {
  __shared__ uint32_t s[K * kMTile];
  __shared__ uint64_t s_split[2];
  __shared__ uint32_t s_prev[2][K];
  __shared__ uint32_t s_hasprev[2];
  __shared__ uint32_t red[kMT / 32 + 1];
  const uint64_t d0 = (uint64_t)blockIdx.x * kMTile;
  const uint64_t d1 = d0 + kMTile < nF + nU ? d0 + kMTile : nF + nU;
  if (threadIdx.x == 0) s_split[0] = merge_split<K>(F, nF, U, nU, d0);
  if (threadIdx.x == 32) s_split[1] = merge_split<K>(F, nF, U, nU, d1);
  __syncthreads();
  const uint64_t a0 = s_split[0], a1 = s_split[1];
  const uint64_t b0 = d0 - a0, b1 = d1 - a1;
  const uint32_t na = (uint32_t)(a1 - a0), nb = (uint32_t)(b1 - b0), nt = na + nb;
  for (uint32_t i = threadIdx.x; i < nt; i += kMT) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      s[k * kMTile + i] = i < na ? __ldg(F.c[k] + a0 + i) : __ldg(U.c[k] + b0 + (i - na));
  }
  if (threadIdx.x == 64) {
    s_hasprev[0] = a0 > 0;
    s_hasprev[1] = b0 > 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      s_prev[0][k] = a0 > 0 ? __ldg(F.c[k] + a0 - 1) : 0u;
      s_prev[1][k] = b0 > 0 ? __ldg(U.c[k] + b0 - 1) : 0u;
    }
  }
  __syncthreads();
  // this thread's share of the tile's merge
  const uint32_t dd = threadIdx.x * kMItems < nt ? threadIdx.x * kMItems : nt;
  uint32_t lo = dd > nb ? dd - nb : 0, hi = dd < na ? dd : na;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (s_le<K>(s, mid, na + (dd - mid - 1)))
      lo = mid + 1;
    else
      hi = mid;
  }
  uint32_t ai = lo, bi = dd - lo;
  uint32_t pf[K], pu[K];
  bool hf, hu;
  if (ai > 0) {
    hf = true;
#pragma unroll
    for (int k = 0; k < K; ++k) pf[k] = s[k * kMTile + ai - 1];
  } else {
    hf = s_hasprev[0];
#pragma unroll
    for (int k = 0; k < K; ++k) pf[k] = s_prev[0][k];
  }
  if (bi > 0) {
    hu = true;
#pragma unroll
    for (int k = 0; k < K; ++k) pu[k] = s[k * kMTile + na + bi - 1];
  } else {
    hu = s_hasprev[1];
#pragma unroll
    for (int k = 0; k < K; ++k) pu[k] = s_prev[1][k];
  }
  uint32_t items[kMItems][K];
  uint32_t has_out = 0, is_new = 0;
  const uint32_t dend = dd + kMItems < nt ? dd + kMItems : nt;
#pragma unroll
  for (int q = 0; q < kMItems; ++q) {
    if (dd + q < dend) {
      const bool take_f = ai < na && (bi >= nb || s_le<K>(s, ai, na + bi));
      if (take_f) {
#pragma unroll
        for (int k = 0; k < K; ++k) items[q][k] = pf[k] = s[k * kMTile + ai];
        hf = true;
        ++ai;
        has_out |= 1u << q;
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) items[q][k] = s[k * kMTile + na + bi];
        const bool rep = (hu && tuple_eq<K>(pu, items[q])) || (hf && tuple_eq<K>(pf, items[q]));
#pragma unroll
        for (int k = 0; k < K; ++k) pu[k] = items[q][k];
        hu = true;
        ++bi;
        if (!rep) {
          has_out |= 1u << q;
          is_new |= 1u << q;
        }
      }
    }
  }
  const uint32_t n_new = __popc(is_new), n_out = __popc(has_out);
  if (!WRITE) {
    uint32_t tot;
    block_exclusive_sum<kMT, uint32_t>(n_new, red, &tot);
    if (threadIdx.x == 0) cnt_out[blockIdx.x] = tot;
    return;
  }
  uint32_t tot_new, tot_out;
  const uint32_t dpos = block_exclusive_sum<kMT, uint32_t>(n_new, red, &tot_new);
  const uint32_t mpos = block_exclusive_sum<kMT, uint32_t>(n_out, red, &tot_out);
  const uint64_t dpre = pre[blockIdx.x];
  // delta straight from registers
#pragma unroll
  for (int q = 0; q < kMItems; ++q) {
    if ((is_new >> q) & 1u) {
      const uint64_t at = dpre + dpos + __popc(is_new & ((1u << q) - 1u));
#pragma unroll
      for (int k = 0; k < K; ++k) D.c[k][at] = items[q][k];
    }
  }
  if (M.c[0] == nullptr) return;
  __syncthreads();  // the tile's inputs are no longer read
#pragma unroll
  for (int q = 0; q < kMItems; ++q) {
    if ((has_out >> q) & 1u) {
      const uint32_t at = mpos + __popc(has_out & ((1u << q) - 1u));
#pragma unroll
      for (int k = 0; k < K; ++k) s[k * kMTile + at] = items[q][k];
    }
  }
  __syncthreads();
  const uint64_t mbase = a0 + dpre;
  for (uint32_t i = threadIdx.x; i < tot_out; i += kMT) {
#pragma unroll
    for (int k = 0; k < K; ++k) M.c[k][mbase + i] = s[k * kMTile + i];
  }
}

template <int K>
cudaError_t run_diff_merge(Ctx& c, ColsIn full, uint64_t n_full, ColsIn fresh, uint64_t n_fresh,
                           ColsOut delta, ColsOut merged, uint64_t* d_ndelta, void* ws) {
  const uint64_t tiles = (n_full + n_fresh + kMTile - 1) / kMTile;
  char* w = static_cast<char*>(ws);
  uint32_t* cnt32 = reinterpret_cast<uint32_t*>(w);
  w += (tiles * 4 + 255) & ~uint64_t(255);
  uint64_t* pre = reinterpret_cast<uint64_t*>(w);
  w += (tiles * 8 + 255) & ~uint64_t(255);
  void* scan_ws = w;
  {
    ProfScope p(c, kDiffCount, 4.0 * K * (n_full + n_fresh));
    k_diff_merge<K, false><<<(unsigned)tiles, kMT, 0, c.st>>>(full, n_full, fresh, n_fresh, cnt32,
                                                             nullptr, delta, merged);
  }
  cudaError_t e = exclusive_scan(c, cnt32, tiles, pre, d_ndelta, scan_ws);
  if (e != cudaSuccess) return e;
  {
    // read Full and New, write Full again; the delta part of the writes
    // (merged and delta) is added once its size is known
    const double mb = merged.c[0] ? 4.0 * K * n_full : 0.0;
    ProfScope p(c, kDiffMerge, 4.0 * K * (n_full + n_fresh) + mb);
    k_diff_merge<K, true><<<(unsigned)tiles, kMT, 0, c.st>>>(full, n_full, fresh, n_fresh, nullptr,
                                                            pre, delta, merged);
  }
  return cudaGetLastError();
}

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

}  // namespace

size_t diff_merge_workspace(uint64_t n_full, uint64_t n_fresh) {
  const uint64_t tiles = (n_full + n_fresh + kMTile - 1) / kMTile;
  return ((tiles * 4 + 255) & ~uint64_t(255)) + ((tiles * 8 + 255) & ~uint64_t(255)) +
         scan_workspace(tiles);
}

cudaError_t diff_merge(Ctx& c, uint32_t k, ColsIn full, uint64_t n_full, ColsIn fresh,
                       uint64_t n_fresh, ColsOut delta, ColsOut merged, uint64_t* d_ndelta,
                       void* ws) {
  if (n_full + n_fresh == 0) return cudaMemsetAsync(d_ndelta, 0, sizeof(uint64_t), c.st);
  switch (k) {
    case 1: return run_diff_merge<1>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws);
    case 2: return run_diff_merge<2>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws);
    case 3: return run_diff_merge<3>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws);
    case 4: return run_diff_merge<4>(c, full, n_full, fresh, n_fresh, delta, merged, d_ndelta, ws);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t select_project(Ctx& c, const SelectSpec& s, ColsOut out, uint64_t* d_cursor,
                           uint64_t out_cap) {
  if (s.n == 0) return cudaSuccess;
  const uint64_t blocks = (s.n + kST * kSItems - 1) / (kST * kSItems);
  ProfScope p(c, kSelect, 4.0 * s.in_k * s.n + 4.0 * s.out_k * s.n);
  k_select<<<(unsigned)blocks, kST, 0, c.st>>>(s, out,
                                               reinterpret_cast<unsigned long long*>(d_cursor),
                                               out_cap, c.d_err);
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
