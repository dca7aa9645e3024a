// Host-side launchers of the round's kernels (internal to libcdl).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace cdl {

// ---------------------------------------------------------------- profiling
// Kernel classes timed separately when the engine runs with timing on.
enum KernelClass : int {
  kHashBuild = 0,
  kCountHeads,
  kJoinCount,
  kScan,
  kJoinWrite,
  kRadixUpsweep,
  kRadixScatter,
  kDiffCount,
  kDiffMerge,
  kSelect,
  kMisc,
  kMlp,
  kJoinDirect,
  kRetire,
  kDense,
  kDedup,
  kNumClasses
};
const char* kernel_class_name(int c);

struct Profiler {
  bool on = false;
  uint32_t mask = ~0u;  // kernel classes timed while on
  struct Rec {
    int cls;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<Rec> open;
  std::vector<cudaEvent_t> pool;
  uint64_t launches[kNumClasses] = {};
  double ms[kNumClasses] = {};
  double bytes[kNumClasses] = {};
  uint64_t total_launches = 0;
  double total_bytes = 0;
  cudaEvent_t get();
  void begin(int cls, cudaStream_t st);
  void end(int cls, double algo_bytes, cudaStream_t st);
  void add_bytes(int cls, double b);  // adds to the latest launch of cls
  void collect();  // waits for recorded events and sums their times
  void reset();
  ~Profiler();
};

// Launch context: stream, device error word, profiler (may be null).
struct Ctx {
  cudaStream_t st = nullptr;
  uint32_t* d_err = nullptr;
  Profiler* prof = nullptr;
  uint64_t spin_limit = 1ull << 26;
  int scan_cls = kScan;  // the class a scan's launches are timed under (a step may own its scans)
};

struct ProfScope {
  Ctx& c;
  int cls;
  double bytes;
  ProfScope(Ctx& ctx, int k, double b) : c(ctx), cls(k), bytes(b) {
    if (c.prof) c.prof->begin(cls, c.st);
  }
  ~ProfScope() {
    if (c.prof) c.prof->end(cls, bytes, c.st);
  }
};

// -------------------------------------------------------------------- hash
uint64_t table_slots(uint64_t n_keys, double load);
// keys: columns k0 (and k1 when non-null) sorted lexicographically, n rows.
cudaError_t hash_build(Ctx& c, const uint32_t* k0, const uint32_t* k1, uint64_t n, Slot* table,
                       uint64_t slots);
// Number of distinct (k0, k1) keys of a sorted column pair into *d_out.
cudaError_t count_heads(Ctx& c, const uint32_t* k0, const uint32_t* k1, uint64_t n,
                        uint64_t* d_out);

// -------------------------------------------------------------------- scan
constexpr int kScanTile = 2048;  // elements per scan tile
size_t scan_workspace(uint64_t n);
// out[i] = sum in[0..i); *d_total = sum of all (device pointer, may be null).
// dn (optional): the actual count in device memory, clamped to n, which
// then only sizes the grid (a launch inside a captured round).
cudaError_t exclusive_scan(Ctx& c, const uint32_t* in, uint64_t n, uint64_t* out,
                           uint64_t* d_total, void* ws, const uint64_t* dn = nullptr);
// Second half of the scan when ws already holds the sums of kScanTile tiles.
cudaError_t scan_finish(Ctx& c, const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* d_total,
                        void* ws, const uint64_t* dn = nullptr);

// -------------------------------------------------------------------- join
struct Ref {
  uint8_t side;  // 0 probe, 1 build, 2 constant, 3 second build side (star joins)
  uint32_t v;
};
struct JoinSpec {
  ColsIn probe;
  uint64_t n_probe;
  uint32_t pk0, pk1;  // probe key columns; pk1 = 0xFF when the key has one word
  ColsIn build;       // sorted by the key columns bk0 (, bk1)
  const Slot* table;
  uint64_t slots;
  uint32_t out_k;
  Ref out[kMaxK];
  uint32_t n_neq;
  Ref neq[4][2];
  uint32_t n_eq;  // extra equalities (join keys beyond two words)
  Ref eq[4][2];
  uint32_t cross;    // 1: no shared variable, every build row matches
  uint32_t n_build;  // build rows (used by cross joins)
  // inside a captured round: the probe columns and row count in device
  // memory (n_probe is then the capacity that sizes the grids); else null
  const ColsIn* dprobe;
  const uint64_t* dn;
  // star join: a second build side, also keyed on probe columns (qk0, qk1;
  // qk1 = 0xFF for one word).  A probe row then matches every pair of a row
  // of its first range and a row of its second (count c1 * c2), the join of
  // the chain's last two atoms with no intermediate table between them.
  uint32_t star;
  uint32_t qk0, qk1;
  ColsIn build2;
  const Slot* table2;
  uint64_t slots2;
};
size_t join_count_workspace(uint64_t n_probe);
// Pass 1 alone: counts[i] for every probe row.
cudaError_t join_count_only(Ctx& c, const JoinSpec& j, uint32_t* counts);
// Pass 1 + 2: counts and exclusive offsets of every probe row; total in *d_total.
cudaError_t join_count_scan(Ctx& c, const JoinSpec& j, uint64_t* d_off, uint64_t* d_total,
                            void* ws);
// Pass 3: writes the output tuples.  With no filters, tuple o goes to
// out[base + o] and *d_cursor grows by total; with filters, survivors are
// packed at *d_cursor (atomic).  out_cap bounds every write.
// ws (optional, join_write_workspace bytes) holds every block's merge-path
// split, computed up front; without it each block searches for its own.
size_t join_write_workspace(uint64_t n_probe, uint64_t total);
// Inside a captured round: d_total (the join size, total then being its
// capacity) comes from device memory; an unfiltered join claims its range
// at *d_cursor first and keeps its start in *d_base (which needs ws); a
// write or claim past out_cap raises *d_soft_err instead of the engine's
// error word.
cudaError_t join_write(Ctx& c, const JoinSpec& j, const uint64_t* d_off, uint64_t total,
                       ColsOut out, uint64_t base, uint64_t* d_cursor, uint64_t out_cap,
                       void* ws, size_t ws_bytes, const uint64_t* d_total = nullptr,
                       uint64_t* d_base = nullptr, uint32_t* d_soft_err = nullptr,
                       const DenseSet* dense = nullptr);
// (dense != null: each output tuple sets its bit in *dense instead of being
// written; out, base, d_cursor and out_cap are then unused.)

// -------------------------------------------------------------- dense sets
// Bits of n rows set in d (a row outside d raises kErrCapacity).
cudaError_t dense_insert(Ctx& c, const DenseSet& d, ColsIn rows, uint64_t n);
size_t dense_extract_workspace(uint64_t nbits);
// The set bits of d as rows in increasing bit order (lexicographic, no
// repeats) into out (cap rows; more raise kErrCapacity); their number in
// *d_count.  Clears d.
cudaError_t dense_extract(Ctx& c, const DenseSet& d, ColsOut out, uint64_t cap,
                          uint64_t* d_count, void* ws);


// -------------------------------------------------------------------- sort
// Digit plan of an LSD radix sort over the packed key of K columns.
struct RadixPlan {
  uint32_t k = 0;
  uint32_t bits = 8;
  uint32_t threads = 512;  // block size of the upsweep and scatter passes (512 or 256)
  uint32_t npass = 0;
  struct Pass {
    uint32_t sh[kMaxK], mask[kMaxK], dsh[kMaxK];
  };
  std::vector<Pass> pass;
};
// Digit width for a key of total_bits: 9 where 9-bit digits take one pass
// fewer than 8-bit ones (36-bit keys: 4 passes instead of 5), else base.
uint32_t fit_digit_bits(uint32_t total_bits, uint32_t base);
// col_bits[k]: significant bits of column k (all values < 2^col_bits[k]).
RadixPlan make_radix_plan(uint32_t k, const uint32_t* col_bits, uint32_t digit_bits,
                          uint32_t threads = 512);
size_t radix_workspace(uint64_t n, uint32_t digit_bits, uint32_t threads = 512);
// Sorts (a, n rows) using b as the alternate buffer; returns in *in_b
// whether the result ended in b.
// dn (optional): the row count in device memory, clamped to n, which then
// only sizes the grids; every pass runs then (none is skipped for one tile).
cudaError_t radix_sort(Ctx& c, const RadixPlan& plan, ColsOut a, ColsOut b, uint64_t n, void* ws,
                       bool* in_b, const uint64_t* dn = nullptr);
// Column maxima into d_max[k] (for plans of unknown data).
cudaError_t column_max(Ctx& c, ColsIn in, uint32_t k, uint64_t n, uint32_t* d_max);

// ------------------------------------------------------- Algorithm 2 dedup
// Full in the decomposed storage model: raw columns in insertion order (row
// = surrogate id); per column k the ids in (value, id) order and the unique
// hashmap over that order (hybrid index), or, hash-only, one multimap of
// (value, id) entries of column 0 (packed as value | id << 32; empty = all
// ones).
struct DsmView {
  ColsIn raw;
  uint64_t n = 0;
  const uint32_t* ids[kMaxK] = {nullptr, nullptr, nullptr, nullptr};
  const Slot* table[kMaxK] = {nullptr, nullptr, nullptr, nullptr};
  uint64_t mask[kMaxK] = {0, 0, 0, 0};
  const uint2* mm = nullptr;
  uint64_t mm_mask = 0;
};
// flags[i] = 1 when sorted row i repeats neither its predecessor nor a row
// of Full (Algorithm 2), else 0.
cudaError_t dsm_probe(Ctx& c, uint32_t k, ColsIn rows, uint64_t n, const DsmView& v,
                      bool hash_only, uint32_t* flags);
// out[off[i]] = rows[i] where flags[i] (off: exclusive scan of flags).
cudaError_t compact_rows(Ctx& c, uint32_t k, ColsIn rows, uint64_t n, const uint32_t* flags,
                         const uint64_t* off, ColsOut out);
// Inserts (keys[i], id0 + i) into the multimap (slots a power of two).
cudaError_t mm_insert(Ctx& c, const uint32_t* keys, uint64_t n, uint32_t id0, uint2* table,
                      uint64_t slots);
// out[i] = first + i.
cudaError_t iota_u32(Ctx& c, uint32_t* out, uint64_t n, uint32_t first);

// ------------------------------------------------------------------ setops
size_t diff_merge_workspace(uint64_t n_full, uint64_t n_fresh);
// A diff_merge inside a captured round: Full's columns and size, the new
// tuples' count and the output columns are read from device memory (n_full
// and n_fresh then only size the grids and clamp the counts).  When |full| +
// |new| exceeds cap_merged nothing is written, |delta| = 0 and *overflow is
// raised.
struct DevMerge {
  const ColsIn* full = nullptr;
  const uint64_t* n_full = nullptr;
  const uint64_t* n_fresh = nullptr;
  const ColsOut* delta = nullptr;
  const ColsOut* merged = nullptr;
  uint64_t cap_merged = 0;
  uint32_t* overflow = nullptr;
};
// delta = fresh - full, merged = full U delta; *d_ndelta receives |delta|.
// When merged.c[0] is null only delta is produced.
cudaError_t diff_merge(Ctx& c, uint32_t k, ColsIn full, uint64_t n_full, ColsIn fresh,
                       uint64_t n_fresh, ColsOut delta, ColsOut merged, uint64_t* d_ndelta,
                       void* ws, const DevMerge* dm = nullptr);

// Selection + projection of one atom: keeps rows with col == const, col ==
// col and (on output refs) out != out; writes out tuples packed at
// *d_cursor (atomic).  Refs use side 0 (input column) or 2 (constant).
struct SelectSpec {
  ColsIn in;
  uint32_t in_k;
  uint64_t n;
  uint32_t n_const;
  uint32_t const_col[kMaxK];
  uint32_t const_val[kMaxK];
  uint32_t n_same;
  uint32_t same[kMaxK][2];
  uint32_t out_k;
  Ref out[kMaxK];
  uint32_t n_neq;
  Ref neq[4][2];
};
// Rows past out_cap are dropped and flagged: kErrCapacity in the error word,
// or *soft_overflow = 1 when soft_overflow is non-null.
cudaError_t select_project(Ctx& c, const SelectSpec& s, ColsOut out, uint64_t* d_cursor,
                           uint64_t out_cap, uint32_t* soft_overflow = nullptr);

// last_round[v] = round for every instance id v < n_instances present in the
// sorted instance column inst (n rows).
// Inside a captured round (dinst non-null): column 0 of *dinst, the count
// *dn (clamped to n) and round + *dround.
cudaError_t mark_instances(Ctx& c, const uint32_t* inst, uint64_t n, uint32_t n_instances,
                           uint64_t* last_round, uint64_t round, const ColsIn* dinst = nullptr,
                           const uint64_t* dn = nullptr, const uint64_t* dround = nullptr);

// ------------------------------------------------------- captured rounds
// Device state of one derived relation in a round captured as a CUDA graph:
// its full and delta versions and their sizes.  A round reads cur and
// writes next; the round's last kernel swaps them.
struct GraphRel {
  ColsIn F, D;
  uint64_t nF, nD;
};
struct GraphCtl {
  uint64_t round;       // rounds completed (all launches, numbered as the engine does)
  uint64_t iterations;  // last round that derived a tuple
  uint64_t done;        // 0 running, 1 fixpoint, 2 a buffer overflowed, 3 past max_iters
  uint64_t max_iters;   // 0: no limit
  uint32_t overflow;    // raised by any launch of the round that ran out of room
  uint32_t pad;
};
// The round's last kernel (one thread): on overflow nothing moves and the
// loop stops (cur still holds the last complete round); else next.nF =
// cur.nF + next.nD, per_round[round] = sum of next.nD, cur <-> next, and the
// loop's condition is set to continue while the round derived something.
// It also zeroes the next round's cursors: `ncur` words at `cursors` and
// every third word from `steps` + 2, `nsteps` of them.
cudaError_t round_end(Ctx& c, GraphRel* cur, GraphRel* next, uint32_t nrel, GraphCtl* ctl,
                      uint64_t* per_round, uint64_t per_round_cap,
                      cudaGraphConditionalHandle loop, uint64_t* cursors, uint32_t ncur,
                      uint64_t* steps, uint32_t nsteps);

// Retirement of converged instances inside a captured batched round (device
// state; retire.cu).  live[i]: instance i's rows are still in Full; conv[i]:
// it reached its fixpoint (rows leave Full, or have left once live is 0).
struct RetireCtl {
  uint32_t* live;
  uint32_t* conv;
  uint32_t go;          // rows move this round
  uint32_t short_room;  // a retired buffer was too small for a move
  uint64_t moves;       // rounds whose converged rows moved out of Full
};
// Per derived relation: the retired rows (instance i: ret_cnt[i] rows from
// ret_off[i]), the instances' bounds in Full, and this round's tables of
// kept and retired segments (one per instance, ni + 1 offsets each).
struct RetireRel {
  ColsOut ret;
  uint64_t ret_cap, ret_n;
  uint64_t* bounds;
  uint64_t* ret_off;
  uint64_t* ret_cnt;
  uint64_t* kseg_off;
  uint64_t* kseg_src;
  uint64_t* rseg_off;
  uint64_t* rseg_src;
  uint64_t kept, moved;
};
// After round_end: converged instances' rows leave cur's Full once they are
// 1/8 of all Full rows (kept rows gathered into next's free Full buffer,
// which then becomes cur's).  arity: host array of the nrel arities.
cudaError_t retire_round(Ctx& c, GraphRel* cur, GraphRel* next, GraphCtl* ctl, RetireCtl* rc,
                         RetireRel* rr, const uint32_t* arity, uint32_t nrel, uint32_t ni,
                         const uint64_t* last_round);
// col[j] = s for the rows j of segment s: [off[s], off[s + 1]), off having
// nseg + 1 device entries and off[nseg] = total.
cudaError_t fill_segments(Ctx& c, uint32_t* col, const uint64_t* off, uint32_t nseg,
                          uint64_t total);
// Segments side by side behind a leading column of segment numbers: row j
// of segment s (rows [off[s], off[s + 1]), off and src in device memory)
// gets out.c[0][j] = s and out.c[1 + c][j] = src[s].c[c][j - off[s]],
// c < k <= 3.
cudaError_t concat_segments(Ctx& c, ColsOut out, const ColsIn* src, uint32_t k,
                            const uint64_t* off, uint32_t nseg, uint64_t total);
// bounds[i] (i = 0..n_instances) = first row of the sorted column inst whose
// value is >= i: instance i occupies rows [bounds[i], bounds[i + 1]).
cudaError_t instance_bounds(Ctx& c, const uint32_t* inst, uint64_t n, uint32_t n_instances,
                            uint64_t* bounds);
// Concatenates nseg row segments of tables a and b (k columns) into out:
// segment s fills out rows [out_off[s], out_off[s + 1]) (out_off has nseg + 1
// entries, out_off[nseg] = total) from row src[s] of a, or of b when bit 63
// of src[s] is set.  All pointers are device pointers.
cudaError_t gather_segments(Ctx& c, uint32_t k, ColsIn a, ColsIn b, const uint64_t* out_off,
                            const uint64_t* src, uint32_t nseg, uint64_t total, ColsOut out);

// Reserved-value check and column maxima of loaded data.
cudaError_t check_values(Ctx& c, ColsIn in, uint32_t k, uint64_t n, uint32_t* d_max);

// ------------------------------------------------------------ estimator
constexpr int kMlpIn = 16, kMlpHidden = 64;
constexpr int kMlpParams = kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden +
                           kMlpHidden + 1;
// Features the host knows about a join (the rest come from key samples).
struct JoinFeatureHost {
  float probe_full;      // size of the full version of the probe relation
  float build_distinct;  // distinct keys of the build side (its index)
  float round;           // semi-naive round
  float prev_output;     // exact output of the same rule step in the previous round
  float prev_delta;      // delta of the head relation in the previous round
  float filtered;        // 1 when the step filters (inequalities, equalities)
};
// workspace of mlp_gradient / mlp_forward for n samples (floats: 4 x 64 n + n)
inline size_t mlp_workspace(uint64_t n) {
  return ((4ull * kMlpHidden * (n ? n : 1) + (n ? n : 1)) * sizeof(float) + 255) & ~size_t(255);
}
cudaError_t mlp_forward(Ctx& c, const float* th, const float* X, uint64_t n, float* out, void* ws);
cudaError_t mlp_gradient(Ctx& c, const float* th, const float* X, const float* y, uint64_t n,
                         float tau, float* out, float* grad, void* ws);
cudaError_t mlp_adam(Ctx& c, float* th, const float* grad, float* m, float* v, uint64_t step,
                     float lr);
cudaError_t mlp_to_bf16(Ctx& c, const float* th, void* tb);
cudaError_t mlp_infer_bf16(Ctx& c, const void* tb, const float* X, uint64_t n, float* out);
cudaError_t join_features(Ctx& c, const uint32_t* pk0, const uint32_t* pk1, uint64_t np,
                          const uint32_t* bk0, const uint32_t* bk1, uint64_t nb,
                          const JoinFeatureHost& hf, float* f);

// Work list of the single-pass join: a probe row whose range holds more
// than kHeavyChunk outputs is cut into chunks of at most kHeavyChunk that
// any warp of a second kernel takes, so one hot key does not serialise a
// warp (the skew Section 4 answers with output partitioning).
constexpr uint32_t kHeavyChunk = 2048;
struct HeavyChunk {
  uint64_t prow;  // probe row
  uint64_t out0;  // first output position (unfiltered joins)
  uint32_t brow;  // first build row of the chunk
  uint32_t len;   // outputs in the chunk
};
struct HeavyList {
  HeavyChunk* e = nullptr;
  uint64_t* n = nullptr;  // device counter, zeroed by the caller
  uint64_t cap = 0;
};

// Single-pass join write sized by a prediction: every probe row claims its
// range at *d_cursor (atomic, one per warp); survivors are written when the
// claim fits below out_cap, else *d_overflow is set and nothing more of that
// warp is written.  *d_total receives the unfiltered join size.  Rows with
// long ranges go through the heavy list (a full list also sets *d_overflow).
cudaError_t join_direct(Ctx& c, const JoinSpec& j, ColsOut out, uint64_t* d_cursor,
                        uint64_t out_cap, uint64_t* d_total, uint32_t* d_overflow,
                        const HeavyList& heavy);

}  // namespace cdl
