// Step (b): the join of Algorithm 1 in three passes.
//
// Pass 1 (count): every probe row looks its key up in the build side's
// hybrid index and stores the matched range length (0 when absent), and
// each tile of rows also sums its lengths -- the first half of the scan.
// Pass 2 (scan): exclusive scan of the lengths into 64-bit output offsets
// (pos_buf) and the total join size (Algorithm 1's reduce).
// Pass 3 (write): output-partitioned, the variant Section 4 chooses for
// skew: each block owns an equal share of the merged sequence of (row
// starts, output positions) -- a merge-path split found by binary search
// over the offsets, so a block's work is bounded whether its rows match
// nothing or one row matches a hundred thousand tuples.  The block re-probes
// the index once per row it covers, then every output position finds its row
// by binary search in shared memory (the search of Algorithm 1's write loop,
// over the non-empty ranges only) and gathers the build row
// start + (n - pos_buf[j]).  Projection, constant head columns, equalities
// beyond the hashed key and inequalities (x != y) are applied in the same
// pass, so the join result is written directly as head columns (Section 4:
// the join result is materialised only at projection).
#include "kernels.h"

namespace cdl {

namespace {

constexpr int kCT = 256;  // count pass: threads; tiles of kScanTile rows
constexpr int kCItems = kScanTile / kCT;
constexpr int kJT = 256;  // write pass threads
constexpr int kDU = 4;    // write pass into a bitmap: outputs per thread in flight
constexpr uint32_t kDRows = 8;  // ... and the most probe rows a block walks one by one
constexpr int kJItems = 8;
constexpr int kJTile = kJT * kJItems;  // merged items per block

// Column v of a column set held in registers: a chain of selects with
// constant indices, so that a run-time column number does not send the set
// to local memory.
__device__ __forceinline__ const uint32_t* col_of(const ColsIn& c, uint32_t v) {
  const uint32_t* p = c.c[0];
#pragma unroll
  for (int k = 1; k < kMaxK; ++k)
    if (v == (uint32_t)k) p = c.c[k];
  return p;
}

__device__ __forceinline__ uint32_t probe_key1(const JoinSpec& j, const ColsIn& probe,
                                              uint64_t row) {
  return j.pk1 == 0xFFu ? 0u : __ldg(col_of(probe, j.pk1) + row);
}

// Range of build rows matching probe row `row`: the hybrid index lookup, or
// every build row for a join without shared variables.
__device__ __forceinline__ uint32_t lookup(const JoinSpec& j, const ColsIn& probe, uint64_t mask,
                                          uint64_t row, uint32_t* start) {
  if (j.cross) {
    *start = 0;
    return j.n_build;
  }
  return probe_table(j.table, mask, __ldg(col_of(probe, j.pk0) + row), probe_key1(j, probe, row),
                     start);
}

// Range of second-build-side rows matching probe row `row` (star joins).
__device__ __forceinline__ uint32_t lookup2(const JoinSpec& j, const ColsIn& probe, uint64_t row,
                                           uint32_t* start) {
  const uint32_t k1 = j.qk1 == 0xFFu ? 0u : __ldg(col_of(probe, j.qk1) + row);
  return probe_table(j.table2, j.slots2 - 1, __ldg(col_of(probe, j.qk0) + row), k1, start);
}

// Output count of probe row `row`: its range length, or for a star join the
// product of its two range lengths (a product past 2^32 - 1 raises
// kErrCapacity and counts 0: no relation holds that many rows).
__device__ __forceinline__ uint32_t row_count(const JoinSpec& j, const ColsIn& probe,
                                             uint64_t mask, uint64_t row, uint32_t* err) {
  uint32_t st;
  const uint32_t c1 = lookup(j, probe, mask, row, &st);
  if (!j.star || c1 == 0) return c1;
  const uint64_t prod = (uint64_t)c1 * lookup2(j, probe, row, &st);
  if (prod > 0xFFFFFFFFull) {
    if (err) atomicOr(err, kErrCapacity);
    return 0;
  }
  return (uint32_t)prod;
}

// The probe side of a launch: the spec's columns and row count, or (inside
// a captured round) the ones device memory holds, the count clamped to the
// capacity the spec's n_probe then gives.
__device__ __forceinline__ ColsIn probe_cols(const JoinSpec& j) {
  return j.dprobe ? *j.dprobe : j.probe;
}

__global__ void __launch_bounds__(kCT) k_join_count(const JoinSpec j, uint32_t* __restrict__ counts,
                                                    uint64_t* __restrict__ tile_sums,
                                                    uint32_t* err) {
  __shared__ uint64_t red[kCT / 32 + 1];
  const uint64_t n = dev_size(j.dn, j.n_probe);
  const ColsIn probe = probe_cols(j);
  const uint64_t mask = j.slots - 1;
  // tile 0 is written even for n == 0; blocks loop over the tiles
  const uint64_t ntiles = n ? (n + kScanTile - 1) / kScanTile : 1;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t base = tile * kScanTile;
    uint64_t s = 0;
#pragma unroll 4
    for (int i = 0; i < kCItems; ++i) {
      const uint64_t row = base + (uint64_t)i * kCT + threadIdx.x;
      if (row < n) {
        const uint32_t cnt = row_count(j, probe, mask, row, err);
        counts[row] = cnt;
        s += cnt;
      }
    }
    uint64_t total;
    block_exclusive_sum<kCT, uint64_t>(s, red, &total);  // ends with a barrier
    if (threadIdx.x == 0) tile_sums[tile] = total;
  }
}

__global__ void __launch_bounds__(kCT) k_join_count_only(const JoinSpec j,
                                                         uint32_t* __restrict__ counts,
                                                         uint32_t* err) {
  const uint64_t row = (uint64_t)blockIdx.x * kCT + threadIdx.x;
  if (row >= j.n_probe) return;
  counts[row] = row_count(j, j.probe, j.slots - 1, row, err);
}

// Number of probe rows among the first d items of the merge of the row
// starts off[0..n) with the output positions 0..total-1 (a row start goes
// before the output positions it is <=).
__device__ __forceinline__ uint64_t merge_split(const uint64_t* off, uint64_t n, uint64_t total,
                                                uint64_t d) {
  uint64_t lo = d > total ? d - total : 0, hi = d < n ? d : n;
  while (lo < hi) {
    const uint64_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(off + mid) <= d - mid - 1)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// All blocks' splits at once, one thread per split, so that no block
// waits on a chain of dependent global loads before its first useful one.
// Inside a captured round an unfiltered join's output range is claimed here
// too (thread 0): *d_base = *cursor, *cursor += the join's size, and a range
// past cap raises *overflow.
__global__ void k_write_splits(const uint64_t* __restrict__ off, uint64_t n, uint64_t total,
                               uint64_t* __restrict__ splits, uint64_t nblocks,
                               const uint64_t* dn, const uint64_t* dtotal,
                               unsigned long long* cursor, uint64_t* d_base, uint64_t cap,
                               uint32_t* overflow) {
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d_base && b == 0) {
    const uint64_t b0 = *cursor, t = *dtotal;
    *d_base = b0;
    *cursor = b0 + t;
    if (b0 + t > cap) atomicOr(overflow, 1u);
  }
  if (dn) {  // sizes from device memory (nblocks was sized for the capacities)
    n = dev_size(dn, n);
    total = dev_size(dtotal, total);
    nblocks = (n + total + kJTile - 1) / kJTile;
  }
  if (b > nblocks) return;
  const uint64_t d = b * kJTile < n + total ? b * kJTile : n + total;
  splits[b] = merge_split(off, n, total, d);
}

__device__ __forceinline__ uint32_t ref_value(const JoinSpec& j, const ColsIn& probe, const Ref& r,
                                              uint64_t row, uint64_t brow, uint64_t brow2 = 0) {
  if (r.side == 0) return __ldg(col_of(probe, r.v) + row);
  if (r.side == 1) return __ldg(j.build.c[r.v] + brow);
  if (r.side == 3) return __ldg(j.build2.c[r.v] + brow2);
  return r.v;
}

// Row heads: five resident blocks per SM (registers capped at 51).  Bitmap
// heads: registers capped at 32, eight blocks per SM (seven for star joins,
// bounded by shared memory); the bit-setting loop is latency-bound, and on
// points-to at 2^-5 this cap took the write from 6.6 s to 5.6 s per
// fixpoint against four or five blocks.
// DENSE: each output tuple sets its bit in dset instead of being written.
// STAR: output n of probe row j (local index l = n - pos_buf[j]) pairs the
// first range's row l / c2 with the second range's row l % c2.
template <bool FILTER, bool DENSE, bool STAR>
__global__ void __launch_bounds__(kJT, DENSE ? 8 : 5) k_join_write(const JoinSpec j, const uint64_t* __restrict__ off,
                                                    uint64_t total, ColsOut out, uint64_t base,
                                                    unsigned long long* cursor, uint64_t out_cap,
                                                    const uint64_t* __restrict__ splits,
                                                    uint32_t* err, const uint64_t* dtotal,
                                                    const uint64_t* dbase, const DenseSet dset) {
  // row r's first output: the carried-in row 0 keeps its global start,
  // every later row starts inside the block's window of at most kJTile
  // outputs and keeps its start relative to the window
  __shared__ uint16_t s_loc[kJTile + 1];
  __shared__ uint64_t s_a0;
  __shared__ uint32_t s_start[kJTile + 1];
  __shared__ uint32_t s_start2[STAR ? kJTile + 1 : 1];  // second range: start, length
  __shared__ uint32_t s_cnt2[STAR ? kJTile + 1 : 1];
  __shared__ uint16_t s_row[DENSE ? 1 : kJTile];  // staged row of each of the block's outputs
  __shared__ uint64_t s_split[2];
  __shared__ uint32_t red[kJT / 32 + 1];
  __shared__ unsigned long long s_base;
  const uint64_t n_probe = dev_size(j.dn, j.n_probe);
  const ColsIn probe = probe_cols(j);
  // a device-given join size past the capacity the launch was sized for:
  // the outputs past it are not written, so the round must be redone (a
  // filtered join's survivors may still have fit: the flag is conservative)
  if (dtotal && blockIdx.x == 0 && threadIdx.x == 0 && *dtotal > total && err)
    atomicOr(err, kErrCapacity);
  total = dev_size(dtotal, total);
  const uint64_t wbase = dbase ? *dbase : base;  // rows of this join start here
  (void)wbase;  // (a bitmap head writes no rows)
  const uint64_t nm = n_probe + total;
  const uint64_t ntiles = (nm + kJTile - 1) / kJTile;  // a device-given size may be below the grid's
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  {
  const uint64_t d0 = tile * kJTile;
  const uint64_t d1 = d0 + kJTile < nm ? d0 + kJTile : nm;
  if (splits) {
    if (threadIdx.x < 2) s_split[threadIdx.x] = splits[tile + threadIdx.x];
  } else {
    if (threadIdx.x == 0) s_split[0] = merge_split(off, n_probe, total, d0);
    if (threadIdx.x == 32) s_split[1] = merge_split(off, n_probe, total, d1);
  }
  // (a device-sized launch had its range claimed by the split kernel)
  if (!FILTER && !DENSE && !dbase && tile == 0 && threadIdx.x == 0)
    atomicAdd(cursor, (unsigned long long)total);
  __syncthreads();
  const uint64_t j0 = s_split[0], j1 = s_split[1];
  const uint64_t o0 = d0 - j0, o1 = d1 - j1;
  const uint64_t r_lo = j0 > 0 ? j0 - 1 : 0;
  const uint32_t nrows = (uint32_t)(j1 - r_lo);
  const uint64_t mask = j.slots - 1;
  // the outputs' rows come from a table where the head is written as rows
  // (a bitmap head's block searches the staged starts, or walks its rows
  // one by one when it has a few: there the table's barriers cost more
  // than the searches they save)
  constexpr bool table = !DENSE;
  const uint32_t no = (uint32_t)(o1 - o0);
  if constexpr (table) {
    for (uint32_t i = threadIdx.x; i < no; i += kJT) s_row[i] = 0;
    __syncthreads();
  }
  for (uint32_t r = threadIdx.x; r < nrows; r += kJT) {
    const uint64_t row = r_lo + r;
    const uint64_t a = __ldg(off + row);
    const uint64_t b = row + 1 < n_probe ? __ldg(off + row + 1) : total;
    uint32_t st = 0;
    if (b > a) lookup(j, probe, mask, row, &st);
    if (r == 0)
      s_a0 = a;
    else
      s_loc[r] = (uint16_t)(a - o0);
    s_start[r] = st;
    // a row with outputs in the block's window marks its first one there
    // (such rows start at distinct outputs; the row carried in from the
    // block before may end at the window's start)
    const uint64_t first = a > o0 ? a : o0;
    if (table && b > first && first < o1) s_row[first - o0] = (uint16_t)r;
    if constexpr (STAR) {
      uint32_t st2 = 0, c2 = 1;
      if (b > a) c2 = lookup2(j, probe, row, &st2);
      s_start2[r] = st2;
      s_cnt2[r] = c2;
    }
  }
  __syncthreads();
  auto off_of = [&](uint32_t r) -> uint64_t { return r == 0 ? s_a0 : o0 + s_loc[r]; };
  // head values of probe row `row` matched with build row `brow`; false
  // when a filter drops the pair
  auto tuple_of = [&](uint64_t row, uint64_t brow, uint64_t brow2,
                      uint32_t (&vals)[kMaxK]) -> bool {
#pragma unroll
    for (int k = 0; k < kMaxK; ++k)
      if (k < (int)j.out_k) vals[k] = ref_value(j, probe, j.out[k], row, brow, brow2);
    bool keep = true;
    if (FILTER) {
      for (uint32_t q = 0; q < j.n_eq; ++q)
        keep &= ref_value(j, probe, j.eq[q][0], row, brow, brow2) ==
                ref_value(j, probe, j.eq[q][1], row, brow, brow2);
      for (uint32_t q = 0; q < j.n_neq; ++q)
        keep &= ref_value(j, probe, j.neq[q][0], row, brow, brow2) !=
                ref_value(j, probe, j.neq[q][1], row, brow, brow2);
    }
    return keep;
  };
  // output l of staged row r (l < its range length, or the product of both)
  auto tuple_in = [&](uint32_t r, uint64_t l, uint32_t (&vals)[kMaxK]) -> bool {
    if constexpr (STAR) {
      const uint32_t c2 = s_cnt2[r];
      const uint32_t l1 = (uint32_t)l / c2;
      return tuple_of(r_lo + r, (uint64_t)s_start[r] + l1,
                      (uint64_t)s_start2[r] + ((uint32_t)l - l1 * c2), vals);
    } else {
      return tuple_of(r_lo + r, (uint64_t)s_start[r] + l, 0, vals);
    }
  };
  // every output takes the last mark at or before it: its row (the
  // load-balanced search of Algorithm 1's write loop, a max-scan over the
  // block's outputs instead of a binary search per output)
  if constexpr (table) {
    const uint32_t q0 = threadIdx.x * kJItems;
    uint16_t loc[kJItems];
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < kJItems; ++q) {
      loc[q] = q0 + q < no ? s_row[q0 + q] : (uint16_t)0;
      m = loc[q] > m ? loc[q] : m;
    }
    uint32_t run = block_exclusive_max<kJT>(m, red);
#pragma unroll
    for (int q = 0; q < kJItems; ++q) {
      run = loc[q] > run ? loc[q] : run;
      if (q0 + q < no) s_row[q0 + q] = (uint16_t)run;
    }
    __syncthreads();
  }
  // output o of the block: its probe row from the table, or the last staged
  // row starting at or before it
  auto tuple_at = [&](uint64_t o, uint32_t (&vals)[kMaxK]) -> bool {
    uint32_t r;
    if constexpr (table) {
      r = s_row[o - o0];
    } else {
      uint32_t lo = 0, hi = nrows;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (o0 + s_loc[mid] <= o)
          lo = mid;
        else
          hi = mid;
      }
      r = lo;
    }
    return tuple_in(r, o - off_of(r), vals);
  };
  if constexpr (DENSE) {
   if (nrows <= kDRows) {
    // a few probe rows with long ranges (the hot keys): the block walks
    // each row's outputs in turn, with no search for the row
    bool bad = false;
    for (uint32_t r = 0; r < nrows; ++r) {
      const uint64_t ra = off_of(r);
      const uint64_t a = ra > o0 ? ra : o0;
      const uint64_t e = r + 1 < nrows ? off_of(r + 1) : o1;
      const uint64_t b = e < o1 ? e : o1;
      for (uint64_t o = a + threadIdx.x; o < b; o += kJT) {
        uint32_t vals[kMaxK] = {0, 0, 0, 0};
        if (!tuple_in(r, o - ra, vals)) continue;
        uint32_t word, bit;
        if (!dense_locate(dset, vals, &word, &bit)) {
          bad = true;
          continue;
        }
        if (dense_missing(dset, word, bit)) atomicOr(dset.words + word, bit);
      }
    }
    if (bad && err) atomicOr(err, kErrCapacity);
   } else {
    // kDU outputs per thread at a time, each stage's loads all in flight:
    // the gathers, the words' reads, the atomics of missing bits
    bool bad = false;
    for (uint64_t ob = o0; ob < o1; ob += (uint64_t)kJT * kDU) {
      uint32_t word[kDU], bit[kDU];
      bool need[kDU];
#pragma unroll
      for (int u = 0; u < kDU; ++u) {
        const uint64_t o = ob + (uint64_t)u * kJT + threadIdx.x;
        uint32_t vals[kMaxK] = {0, 0, 0, 0};
        word[u] = bit[u] = 0;
        need[u] = o < o1 && tuple_at(o, vals);
        if (need[u] && !dense_locate(dset, vals, &word[u], &bit[u])) bad = true, need[u] = false;
      }
#pragma unroll
      for (int u = 0; u < kDU; ++u)
        if (need[u]) need[u] = dense_missing(dset, word[u], bit[u]);
#pragma unroll
      for (int u = 0; u < kDU; ++u)
        if (need[u]) atomicOr(dset.words + word[u], bit[u]);
    }
    if (bad && err) atomicOr(err, kErrCapacity);
   }
  }
  if constexpr (!DENSE)
  for (uint64_t ob = o0; ob < o1; ob += kJT) {
    const uint64_t o = ob + threadIdx.x;
    const bool valid = o < o1;
    uint32_t vals[kMaxK] = {0, 0, 0, 0};
    const bool keep = valid && tuple_at(o, vals);
    uint64_t pos;
    if (FILTER) {
      uint32_t cnt;
      const uint32_t local = block_exclusive_sum<kJT, uint32_t>(keep ? 1u : 0u, red, &cnt);
      if (threadIdx.x == 0) s_base = cnt ? atomicAdd(cursor, (unsigned long long)cnt) : 0ull;
      __syncthreads();
      pos = s_base + local;
      __syncthreads();
    } else {
      pos = wbase + o;
    }
    if (keep) {
      if (pos < out_cap) {
#pragma unroll
        for (int k = 0; k < kMaxK; ++k)
          if (k < (int)j.out_k) out.c[k][pos] = vals[k];
      } else {
        if (err) atomicOr(err, kErrCapacity);
      }
    }
  }
  }
  __syncthreads();  // the next tile restages the offsets and splits
  }
}

}  // namespace

cudaError_t join_count_only(Ctx& c, const JoinSpec& j, uint32_t* counts) {
  if (j.n_probe == 0) return cudaSuccess;
  ProfScope p(c, kJoinCount, (j.pk1 == 0xFFu ? 4.0 : 8.0) * j.n_probe + 20.0 * j.n_probe);
  k_join_count_only<<<(unsigned)((j.n_probe + kCT - 1) / kCT), kCT, 0, c.st>>>(j, counts,
                                                                              c.d_err);
  return cudaGetLastError();
}

size_t join_count_workspace(uint64_t n_probe) {
  const size_t counts = ((n_probe * sizeof(uint32_t)) + 255) & ~size_t(255);
  return counts + scan_workspace(n_probe);
}

cudaError_t join_count_scan(Ctx& c, const JoinSpec& j, uint64_t* d_off, uint64_t* d_total,
                            void* ws) {
  if (j.n_probe == 0) return cudaMemsetAsync(d_total, 0, sizeof(uint64_t), c.st);
  uint32_t* counts = static_cast<uint32_t*>(ws);
  void* scan_ws = static_cast<char*>(ws) + (((j.n_probe * sizeof(uint32_t)) + 255) & ~size_t(255));
  const uint64_t tiles = (j.n_probe + kScanTile - 1) / kScanTile;
  {
    // per row: its key, the slot probed, the count written (a star join's
    // second key and slot are read for rows its first range matches)
    double keyb = j.pk1 == 0xFFu ? 4.0 : 8.0;
    if (j.star) keyb += (j.qk1 == 0xFFu ? 4.0 : 8.0) + 16.0;
    ProfScope p(c, kJoinCount, (keyb + 16.0 + 4.0) * j.n_probe);
    k_join_count<<<dev_grid(tiles, j.dn), kCT, 0, c.st>>>(j, counts,
                                                           static_cast<uint64_t*>(scan_ws), c.d_err);
  }
  return scan_finish(c, counts, j.n_probe, d_off, d_total, scan_ws, j.dn);
}

// ------------------------------------------------------------ single pass
// The write without count and scan, for joins sized by the estimator: a
// block takes 256 probe rows at a time, scans their range lengths in shared
// memory, claims the rows' outputs with one atomic on the cursor and writes
// them together -- thread t writes outputs t, t + 256, ..., each finding its
// row by binary search over the block's offsets, as the exact write does.
// A row with more than kHeavyChunk outputs goes to the heavy list instead,
// so a hot key never holds one block.
constexpr int kDirT = 256;

// Writes the outputs [o_begin, o_end) of probe row prow (build rows from
// brow0) as one warp: unfiltered outputs go to pos0 + o, filtered ones are
// packed with a ballot and one cursor claim per 32.
template <bool FILTER>
__device__ __forceinline__ void warp_emit(const JoinSpec& j, ColsOut out, uint64_t prow,
                                          uint64_t brow0, uint64_t len, uint64_t pos0,
                                          unsigned long long* cursor, uint64_t cap,
                                          uint32_t* overflow) {
  const uint32_t lane = lane_id();
  const uint32_t lt = lanemask_lt();
  for (uint64_t ob = 0; ob < len; ob += 32) {
    const uint64_t o = ob + lane;
    const bool valid = o < len;
    uint32_t vals[kMaxK] = {0, 0, 0, 0};
    bool keep = valid;
    if (valid) {
#pragma unroll
      for (int k = 0; k < kMaxK; ++k)
        if (k < (int)j.out_k) vals[k] = ref_value(j, j.probe, j.out[k], prow, brow0 + o);
      if (FILTER) {
        for (uint32_t q = 0; q < j.n_eq; ++q)
          keep &= ref_value(j, j.probe, j.eq[q][0], prow, brow0 + o) ==
                  ref_value(j, j.probe, j.eq[q][1], prow, brow0 + o);
        for (uint32_t q = 0; q < j.n_neq; ++q)
          keep &= ref_value(j, j.probe, j.neq[q][0], prow, brow0 + o) !=
                  ref_value(j, j.probe, j.neq[q][1], prow, brow0 + o);
      }
    }
    uint64_t pos;
    if (FILTER) {
      const uint32_t bal = __ballot_sync(0xffffffffu, keep);
      uint64_t cb = 0;
      if (lane == 0 && bal) cb = atomicAdd(cursor, (unsigned long long)__popc(bal));
      cb = __shfl_sync(0xffffffffu, cb, 0);
      pos = cb + __popc(bal & lt);
      if (bal && cb + __popc(bal) > cap && lane == 0) atomicOr(overflow, 1u);
    } else {
      pos = pos0 + o;
    }
    if (keep && pos < cap) {
#pragma unroll
      for (int k = 0; k < kMaxK; ++k)
        if (k < (int)j.out_k) out.c[k][pos] = vals[k];
    }
  }
}

template <bool FILTER>
__global__ void __launch_bounds__(kDirT) k_join_direct(const JoinSpec j, ColsOut out,
                                                       unsigned long long* cursor, uint64_t cap,
                                                       unsigned long long* total,
                                                       uint32_t* overflow, HeavyList heavy) {
  __shared__ uint32_t s_off[kDirT];    // block-local exclusive offsets of the rows
  __shared__ uint32_t s_start[kDirT];  // first build row of each row's range
  __shared__ uint32_t red[kDirT / 32 + 1];
  __shared__ unsigned long long s_base;
  const uint64_t mask = j.slots - 1;
  for (uint64_t b0 = (uint64_t)blockIdx.x * kDirT; b0 < j.n_probe;
       b0 += (uint64_t)gridDim.x * kDirT) {
    const uint64_t row = b0 + threadIdx.x;
    uint32_t st = 0, cnt = 0;
    if (row < j.n_probe) cnt = lookup(j, j.probe, mask, row, &st);
    if (cnt > kHeavyChunk) {  // a long range becomes chunks of the heavy list
      atomicAdd(total, (unsigned long long)cnt);
      uint64_t out0 = 0;
      bool ok = true;
      if (!FILTER) {
        out0 = atomicAdd(cursor, (unsigned long long)cnt);
        ok = out0 + cnt <= cap;
      }
      const uint32_t nch = (cnt + kHeavyChunk - 1) / kHeavyChunk;
      const uint64_t at = ok ? atomicAdd((unsigned long long*)heavy.n, (unsigned long long)nch) : 0;
      ok &= at + nch <= heavy.cap;
      if (ok) {
        for (uint32_t q = 0; q < nch; ++q) {
          HeavyChunk h;
          h.prow = row;
          h.out0 = out0 + (uint64_t)q * kHeavyChunk;
          h.brow = st + q * kHeavyChunk;
          h.len = q + 1 < nch ? kHeavyChunk : cnt - q * kHeavyChunk;
          heavy.e[at + q] = h;
        }
      } else {
        atomicOr(overflow, 1u);
      }
      cnt = 0;
    }
    uint32_t tot;
    const uint32_t ex = block_exclusive_sum<kDirT, uint32_t>(cnt, red, &tot);
    s_off[threadIdx.x] = ex;
    s_start[threadIdx.x] = st;
    if (threadIdx.x == 0 && tot) {
      atomicAdd(total, (unsigned long long)tot);
      if (!FILTER) {
        s_base = atomicAdd(cursor, (unsigned long long)tot);
        if (s_base + tot > cap) atomicOr(overflow, 1u);
      }
    }
    __syncthreads();
    if (tot == 0) continue;  // uniform: nothing of this block reads s_off
    for (uint32_t ob = 0; ob < tot; ob += kDirT) {
      const uint32_t o = ob + threadIdx.x;
      const bool valid = o < tot;
      uint32_t vals[kMaxK] = {0, 0, 0, 0};
      bool keep = valid;
      if (valid) {
        uint32_t lo = 0, hi = kDirT;  // the last row whose range starts at or before o
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (s_off[mid] <= o)
            lo = mid;
          else
            hi = mid;
        }
        const uint64_t prow = b0 + lo;
        const uint64_t brow = (uint64_t)s_start[lo] + (o - s_off[lo]);
#pragma unroll
        for (int k = 0; k < kMaxK; ++k)
          if (k < (int)j.out_k) vals[k] = ref_value(j, j.probe, j.out[k], prow, brow);
        if (FILTER) {
          for (uint32_t q = 0; q < j.n_eq; ++q)
            keep &= ref_value(j, j.probe, j.eq[q][0], prow, brow) ==
                    ref_value(j, j.probe, j.eq[q][1], prow, brow);
          for (uint32_t q = 0; q < j.n_neq; ++q)
            keep &= ref_value(j, j.probe, j.neq[q][0], prow, brow) !=
                    ref_value(j, j.probe, j.neq[q][1], prow, brow);
        }
      }
      uint64_t pos;
      if (FILTER) {  // survivors packed with one claim per 256 outputs
        uint32_t n_keep;
        const uint32_t local = block_exclusive_sum<kDirT, uint32_t>(keep ? 1u : 0u, red, &n_keep);
        if (threadIdx.x == 0) {
          s_base = n_keep ? atomicAdd(cursor, (unsigned long long)n_keep) : 0ull;
          if (n_keep && s_base + n_keep > cap) atomicOr(overflow, 1u);
        }
        __syncthreads();
        pos = s_base + local;
        __syncthreads();
      } else {
        pos = s_base + o;
      }
      if (keep && pos < cap) {
#pragma unroll
        for (int k = 0; k < kMaxK; ++k)
          if (k < (int)j.out_k) out.c[k][pos] = vals[k];
      }
    }
    __syncthreads();  // s_off, s_start and s_base are rewritten by the next rows
  }
}

// The heavy list: one warp per chunk, grid-stride over the chunks the
// direct kernel listed (their number is read from device memory).
template <bool FILTER>
__global__ void __launch_bounds__(kDirT) k_join_heavy(const JoinSpec j, ColsOut out,
                                                      unsigned long long* cursor, uint64_t cap,
                                                      uint32_t* overflow, HeavyList heavy) {
  const uint64_t nwarps = ((uint64_t)gridDim.x * kDirT) >> 5;
  uint64_t n = *heavy.n;
  if (n > heavy.cap) n = heavy.cap;
  for (uint64_t w = ((uint64_t)blockIdx.x * kDirT + threadIdx.x) >> 5; w < n; w += nwarps) {
    const HeavyChunk h = heavy.e[w];
    warp_emit<FILTER>(j, out, h.prow, h.brow, h.len, h.out0, cursor, cap, overflow);
  }
}

cudaError_t join_direct(Ctx& c, const JoinSpec& j, ColsOut out, uint64_t* d_cursor,
                        uint64_t out_cap, uint64_t* d_total, uint32_t* d_overflow,
                        const HeavyList& heavy) {
  if (j.star) return cudaErrorInvalidValue;  // star joins keep the count pass
  if (j.n_probe == 0) return cudaSuccess;
  uint64_t blocks = (j.n_probe + kDirT - 1) / kDirT;
  if (blocks > 152 * 8) blocks = 152 * 8;
  const bool filter = j.n_neq > 0 || j.n_eq > 0;
  ProfScope p(c, kJoinDirect, (4.0 + 16.0 + 4.0 * j.out_k) * j.n_probe);
  auto* cur = reinterpret_cast<unsigned long long*>(d_cursor);
  auto* tot = reinterpret_cast<unsigned long long*>(d_total);
  if (filter) {
    k_join_direct<true><<<(unsigned)blocks, kDirT, 0, c.st>>>(j, out, cur, out_cap, tot, d_overflow,
                                                              heavy);
    k_join_heavy<true><<<152 * 8, kDirT, 0, c.st>>>(j, out, cur, out_cap, d_overflow, heavy);
  } else {
    k_join_direct<false><<<(unsigned)blocks, kDirT, 0, c.st>>>(j, out, cur, out_cap, tot,
                                                               d_overflow, heavy);
    k_join_heavy<false><<<152 * 8, kDirT, 0, c.st>>>(j, out, cur, out_cap, d_overflow, heavy);
  }
  return cudaGetLastError();
}

size_t join_write_workspace(uint64_t n_probe, uint64_t total) {
  const uint64_t blocks = (n_probe + total + kJTile - 1) / kJTile;
  return ((blocks + 1) * 8 + 255) & ~uint64_t(255);
}

cudaError_t join_write(Ctx& c, const JoinSpec& j, const uint64_t* d_off, uint64_t total,
                       ColsOut out, uint64_t base, uint64_t* d_cursor, uint64_t out_cap,
                       void* ws, size_t ws_bytes, const uint64_t* d_total, uint64_t* d_base,
                       uint32_t* d_soft_err, const DenseSet* dense) {
  if (total == 0 || j.n_probe == 0) return cudaSuccess;
  const uint64_t nm = j.n_probe + total;
  const uint64_t blocks = (nm + kJTile - 1) / kJTile;
  const bool filter = j.n_neq > 0 || j.n_eq > 0;
  uint64_t* splits = nullptr;
  if (ws && ws_bytes >= join_write_workspace(j.n_probe, total)) {
    splits = static_cast<uint64_t*>(ws);
    k_write_splits<<<(unsigned)((blocks + 1 + 255) / 256), 256, 0, c.st>>>(
        d_off, j.n_probe, total, splits, blocks, j.dn, d_total,
        reinterpret_cast<unsigned long long*>(d_cursor), d_base, out_cap,
        d_soft_err ? d_soft_err : c.d_err);
  }
  // per probe row: two offsets, key, re-probed slot (a star join: both
  // keys and slots), its own head columns; per output: the gathered build
  // columns and the written head columns
  uint32_t nbuild = 0, nprobe = 0;
  for (uint32_t k = 0; k < j.out_k; ++k) {
    nbuild += j.out[k].side == 1 || j.out[k].side == 3;
    nprobe += j.out[k].side == 0;
  }
  const double row_b = j.star ? 16.0 + 8.0 + 32.0 : 16.0 + 4.0 + 16.0;
  // (a dense head's bits are set in L2-resident words, not written out)
  const double bytes = (row_b + 4.0 * nprobe) * j.n_probe +
                       (4.0 * nbuild + (dense ? 0.0 : 4.0 * j.out_k)) * total;
  ProfScope p(c, kJoinWrite, bytes);
  auto* cur = reinterpret_cast<unsigned long long*>(d_cursor);
  uint32_t* err = d_soft_err ? d_soft_err : c.d_err;
  const DenseSet ds = dense ? *dense : DenseSet{};
  const unsigned grid = dev_grid(blocks, d_total);
#define CDL_JOIN_WRITE(F, D, S)                                                          \
  k_join_write<F, D, S><<<grid, kJT, 0, c.st>>>(j, d_off, total, out, base, cur, out_cap, \
                                                splits, err, d_total, d_base, ds)
  if (j.star) {
    if (dense && filter) CDL_JOIN_WRITE(true, true, true);
    else if (dense) CDL_JOIN_WRITE(false, true, true);
    else if (filter) CDL_JOIN_WRITE(true, false, true);
    else CDL_JOIN_WRITE(false, false, true);
  } else {
    if (dense && filter) CDL_JOIN_WRITE(true, true, false);
    else if (dense) CDL_JOIN_WRITE(false, true, false);
    else if (filter) CDL_JOIN_WRITE(true, false, false);
    else CDL_JOIN_WRITE(false, false, false);
  }
#undef CDL_JOIN_WRITE
  return cudaGetLastError();
}

}  // namespace cdl
