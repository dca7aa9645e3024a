// The semi-naive fixpoint engine behind the C ABI (include/cdl.h).
//
// Host side of the method: relations as uint32 columns in device memory
// (Section 3), rules lowered to copy / join / project plans over them
// (Section 4), and the round loop of semi-naive evaluation with full, delta
// and new versions, every rule applied once per round and one merge per
// derived relation per round (Section 3).  Every step of a round runs in the
// kernels of hash.cu, join.cu, scan.cu, sort.cu and setops.cu; the host only
// plans, allocates and reads back the sizes it needs to size the next launch.
//
// Round r > 1 evaluates, for every rule and every body atom i over a derived
// relation, the variant that reads delta_{r-1} at atom i and the full
// relation at every other atom.  (The textbook variant reads full - delta at
// the atoms before i; reading full instead derives a superset of the same
// tuples, and the difference with full removes the extra ones, so the
// delta of every round is unchanged.)  Round 1 applies every rule to the
// loaded facts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/cdl.h"
#include "kernels.h"
#include "tuner.h"

using namespace cdl;

namespace {

// ----------------------------------------------------------------- memory
// Best-fit sub-allocator over chunks obtained from the caller's allocator
// (or cudaMalloc).  Every kernel of an engine runs on one stream, so a block
// freed here can be handed to the next launch without a synchronisation.
class Pool {
 public:
  cdl_alloc_fn af = nullptr;
  cdl_free_fn ff = nullptr;
  void* ctx = nullptr;
  uint64_t limit = 0;
  uint64_t held = 0;
  // chunks of pinned host memory the GPU reads and writes directly (over
  // the CPU-GPU link) instead of device memory: relations kept out of HBM
  bool host = false;

  void* get(size_t bytes) {
    bytes = bytes ? (bytes + 255) & ~size_t(255) : 256;
    auto it = by_size_.lower_bound(bytes);
    if (it == by_size_.end()) {
      if (!grow(bytes)) return nullptr;
      it = by_size_.lower_bound(bytes);
      if (it == by_size_.end()) return nullptr;
    }
    char* p = it->second;
    size_t sz = it->first;
    by_size_.erase(it);
    Block b = free_[p];
    free_.erase(p);
    if (sz - bytes >= 256) {
      free_[p + bytes] = Block{sz - bytes, b.chunk};
      by_size_.emplace(sz - bytes, p + bytes);
      sz = bytes;
    }
    used_[p] = Block{sz, b.chunk};
    return p;
  }

  void put(void* vp) {
    char* p = static_cast<char*>(vp);
    auto it = used_.find(p);
    if (it == used_.end()) return;
    Block b = it->second;
    used_.erase(it);
    auto nx = free_.find(p + b.size);
    if (nx != free_.end() && nx->second.chunk == b.chunk) {
      erase_size(nx->first, nx->second.size);
      b.size += nx->second.size;
      free_.erase(nx);
    }
    auto pv = free_.lower_bound(p);
    if (pv != free_.begin()) {
      --pv;
      if (pv->first + pv->second.size == p && pv->second.chunk == b.chunk) {
        erase_size(pv->first, pv->second.size);
        pv->second.size += b.size;
        by_size_.emplace(pv->second.size, pv->first);
        return;
      }
    }
    free_[p] = b;
    by_size_.emplace(b.size, p);
  }

  // Returns every chunk with nothing allocated in it to the allocator.
  void trim() {
    for (auto it = chunks_.begin(); it != chunks_.end();) {
      auto f = free_.find(it->first);
      if (f != free_.end() && f->second.size == it->second) {
        erase_size(f->first, f->second.size);
        free_.erase(f);
        release(it->first, it->second);
        held -= it->second;
        it = chunks_.erase(it);
      } else {
        ++it;
      }
    }
  }

  void release_all() {
    for (auto& c : chunks_) release(c.first, c.second);
    chunks_.clear();
    free_.clear();
    by_size_.clear();
    used_.clear();
    held = 0;
  }

 private:
  struct Block {
    size_t size;
    char* chunk;  // base of the chunk the block lies in
  };
  std::map<char*, size_t> chunks_;
  std::map<char*, Block> free_;
  std::multimap<size_t, char*> by_size_;
  std::unordered_map<char*, Block> used_;

  void release(char* p, size_t bytes) {
    if (host)
      cudaFreeHost(p);
    else if (ff)
      ff(p, bytes, ctx);
    else
      cudaFree(p);
  }

  void* acquire(size_t want) {
    void* p = nullptr;
    if (host) {
      if (cudaHostAlloc(&p, want, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
      }
    } else if (af) {
      p = af(want, ctx);
    } else if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return p;
  }

  // A new chunk; chunks with nothing in them are returned first so that a
  // growing relation reuses the memory of its previous, smaller version.
  bool grow(size_t bytes) {
    trim();
    size_t want = std::max(bytes, size_t(64) << 20);
    // pinning host memory costs far more than a device allocation: host
    // chunks grow geometrically, so a relation growing every round pins
    // O(log) times
    if (host) want = std::max(bytes * 2, size_t(1) << 30);
    if (limit && held + want > limit) {
      want = bytes;
      if (held + want > limit) return false;
    }
    void* p = acquire(want);
    if (!p && want > bytes) {
      want = bytes;
      p = acquire(want);
    }
    if (!p) return false;
    char* c = static_cast<char*>(p);
    chunks_[c] = want;
    held += want;
    free_[c] = Block{want, c};
    by_size_.emplace(want, c);
    return true;
  }
  void erase_size(char* p, size_t sz) {
    auto r = by_size_.equal_range(sz);
    for (auto i = r.first; i != r.second; ++i)
      if (i->second == p) {
        by_size_.erase(i);
        return;
      }
  }
};

struct DBuf {
  Pool* pool = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { swap(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      reset();
      swap(o);
    }
    return *this;
  }
  ~DBuf() { reset(); }
  void reset() {
    if (pool && p) pool->put(p);
    p = nullptr;
    bytes = 0;
  }
  void swap(DBuf& o) {
    std::swap(pool, o.pool);
    std::swap(p, o.p);
    std::swap(bytes, o.bytes);
  }
};

// A relation version or a temporary table: k device columns of cap rows.
struct DCols {
  DBuf buf;
  uint32_t k = 0;
  uint64_t n = 0, cap = 0;
  uint32_t* c[kMaxK] = {nullptr, nullptr, nullptr, nullptr};
  ColsIn in() const {
    ColsIn r;
    for (int i = 0; i < kMaxK; ++i) r.c[i] = c[i];
    return r;
  }
  ColsOut out() const {
    ColsOut r;
    for (int i = 0; i < kMaxK; ++i) r.c[i] = c[i];
    return r;
  }
  void clear() {
    buf.reset();
    n = cap = 0;
    for (auto& p : c) p = nullptr;
  }
};

size_t col_stride(uint64_t cap) { return ((cap ? cap : 1) * 4 + 255) & ~uint64_t(255); }

uint32_t bits_of(uint64_t v) {
  uint32_t b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

enum Ver { kFull = 0, kDelta = 1 };

// Full of a derived relation in the decomposed storage model, for the
// Algorithm 2 form of step (d) (option dedup; kernels in dsm.cu): rows in
// insertion order (row = surrogate id), and per column k its sorted index,
// kept as (value, id) pairs in (value, id) order, with the unique hashmap
// over the values (dedup 1), or one multimap of column 0's (value, id)
// entries (dedup 2).  Each round appends delta to the rows, merges delta's
// entries into each column's sorted index and rebuilds the hashmaps.
struct Dsm {
  bool on = false;    // the relation's step (d) is Algorithm 2
  bool init = false;  // built from the relation's rows at its first merge
  DCols raw;          // rows in insertion order; raw.n rows
  DCols idx[kMaxK];   // column k: c[0] values ascending, c[1] ids (ascending per value)
  DBuf table[kMaxK];  // column k's unique hashmap over idx[k].c[0]
  uint64_t slots[kMaxK] = {0, 0, 0, 0};
  DBuf mm;            // hash-only: multimap of column 0
  uint64_t mm_slots = 0;
  void reset() {
    on = init = false;
    raw.clear();
    for (int k = 0; k < kMaxK; ++k) {
      idx[k].clear();
      table[k].reset();
      slots[k] = 0;
    }
    mm.reset();
    mm_slots = 0;
  }
};

struct Relation {
  std::string name;
  uint32_t arity = 0;
  bool idb = false;
  DCols full, delta, fresh;
  std::vector<DCols> pending;  // checked loads not yet sorted into full
  uint64_t fresh_ub = 0;
  bool fresh_overflow = false;  // a predicted join of this round claimed past fresh.cap
  uint32_t bound[kMaxK] = {0, 0, 0, 0};  // every value of column k is <= bound[k]
  uint64_t version[2] = {1, 1};
  uint64_t delta_version = 0;  // the Full version the last merge made: Full = previous Full + delta
  bool host_full = false;      // Full kept in pinned host memory (option host_full)
  // batched runs: the rows of instances that reached their fixpoint leave
  // full for this buffer (instance i: ret_cnt[i] rows from ret_off[i])
  DCols retired;
  std::vector<uint64_t> ret_off, ret_cnt;
  // dense form (a tuple space of at most 2^dense_bits): the hash joins of a
  // round set the bits of their tuples in dset; at the round's end the rows
  // written to fresh join them, and dense_rows takes the bits back out as
  // sorted unique rows
  DenseSet dset{};
  DBuf dset_buf;
  uint64_t dense_ub = 0;  // tuples sent to dset this round: a bound on its bits
  DCols dense_rows;
  Dsm dsm;
};

struct Term {
  bool is_const;
  uint32_t v;
};
struct AtomR {
  uint32_t rel;
  std::vector<Term> t;
};
struct RuleR {
  AtomR head;
  std::vector<AtomR> body;
  std::vector<std::pair<uint32_t, uint32_t>> neq;
};

// A hybrid index: the version's tuples sorted by the key columns first and
// the hash table over the distinct keys.
struct Index {
  int rel = -1, ver = -1;
  uint64_t version = 0;
  std::vector<uint32_t> key;
  DCols sorted;  // unused when the relation's own order already starts with the key
  const uint32_t* cols[kMaxK] = {nullptr, nullptr, nullptr, nullptr};  // original numbering
  uint64_t n = 0;
  DBuf table;
  uint64_t slots = 0;
  uint64_t distinct = 0;  // distinct keys
  std::string tkey;       // tuner decision of the load factor, if any
  int tcand = 0;
};

// A table the join chain reads: columns hold the listed variables.
struct Src {
  const uint32_t* c[kMaxK] = {nullptr, nullptr, nullptr, nullptr};
  uint64_t n = 0;
  uint32_t k = 0;
  std::vector<uint32_t> vars;
  std::vector<uint32_t> bits;
  int rel = -1, ver = -1;  // a relation version's own columns, else -1
  DCols owned;
  ColsIn in() const {
    ColsIn r;
    for (int i = 0; i < kMaxK; ++i) r.c[i] = c[i];
    return r;
  }
};

constexpr uint32_t kMaxRels = 1024;
// control block slots (uint64): 0 error word, 1 scratch, 2 aux cursor,
// 3 single-pass join size, 4 overflow flag, 5 overflow flag of the round's
// deferred checks, 8 + r fresh cursor of relation r,
// 8 + kMaxRels + r delta size of relation r
constexpr uint32_t kSlotErr = 0, kSlotScratch = 1, kSlotAux = 2, kSlotDirTotal = 3,
                   kSlotOverflow = 4, kSlotRoundOverflow = 5, kSlotCursor = 8,
                   kSlotDelta = 8 + kMaxRels,
                   kCtlSlots = 8 + 2 * kMaxRels;
constexpr int kEstFloats = 32;  // 16 features, the prediction, padding

}  // namespace

struct cdl_engine {
  cdl_options opt{};
  cudaStream_t st = nullptr;
  Pool pool;
  Pool hpool;  // pinned host memory for relations kept out of device memory (option host_full)
  Profiler prof;
  Ctx ctx;
  std::string err;
  std::vector<std::unique_ptr<Relation>> rels;
  std::map<std::string, uint32_t> by_name;
  std::vector<RuleR> rules;
  bool ran = false;
  DBuf ctl;
  uint64_t* h_ctl = nullptr;
  std::vector<std::unique_ptr<Index>> cache;
  // indexes of a Full version sorted by non-leading key columns, kept one
  // round past their version: the next version's index is this one merged
  // with the round's delta (incremental maintenance) instead of a new sort
  std::vector<std::unique_ptr<Index>> prev_full;
  uint64_t index_merges = 0;
  uint64_t star_joins = 0;  // joins that probed two build sides from one probe row
  uint32_t radix_bits = 0;  // digit width 8, 9 or 10; 0: 8, or 9 where that saves a pass
  uint32_t digits_for(uint32_t total_bits) const {
    return radix_bits ? radix_bits : fit_digit_bits(total_bits, 8);
  }
  double hash_load = 0.5;
  Tuner tuner;
  uint64_t joins = 0;
  // learned join-size estimator
  DBuf est_w, est_wb, est_io;  // FP32 and BF16 parameters; features + prediction
  float* h_est = nullptr;      // pinned host mirror of est_io
  // A round's predictions for its first joins that write a head relation,
  // computed together: a planning pass over the rules launches their
  // features (est_plan), one inference and one read-back follow, and the
  // joins then run without a wait each.
  static constexpr uint32_t kEstBatch = 1024;
  DBuf est_bio;              // kEstBatch x kMlpIn features, then kEstBatch predictions
  float* h_batch = nullptr;  // pinned host mirror of est_bio
  bool est_plan = false;
  uint32_t est_nb = 0;
  std::map<std::tuple<size_t, size_t, size_t>, uint32_t> est_slot;
  bool est_weights = false;
  double est_margin = 1.0;  // the configured margin (log2 units)
  double est_boost = 0.0;   // added after each overrun of this run, up to 4
  uint64_t est_pred = 0, est_over = 0;
  uint64_t cur_round = 0;
  std::vector<float> log_x, log_y;
  std::map<std::tuple<size_t, size_t, size_t>, uint64_t> prev_out;
  // predicted joins that write a head relation leave their overflow check
  // to the end of the round: their sizes land in join_sizes[i]
  static constexpr uint32_t kMaxDeferred = 4096;
  static constexpr double kDirectMaxTuples = double(1 << 24);
  static constexpr uint64_t kPredictMinRows = 1 << 15;  // smaller probes keep the count pass
  static constexpr int kDenseBits = 28;  // default bound of a dense relation's tuple space (32 MB)
  static constexpr int kDenseBitsMax = 34;  // largest bitmap form accepted (2 GB per relation)
  static constexpr uint64_t kGroupRows = 1 << 21;  // larger new-tuple sets sort on their own
  static constexpr size_t kGroupMin = 4;           // fewer relations sort one by one
  struct Deferred {
    std::tuple<size_t, size_t, size_t> step;
    uint32_t head = 0;  // relation the join appends to
    float feat[kMlpIn];
  };
  std::vector<Deferred> deferred;
  DBuf join_sizes;
  DBuf heavy_buf;  // the single-pass join's list of long-range chunks
  HeavyList heavy;
  bool force_exact = false;  // rules are being redone without predictions
  // rounds captured as a CUDA graph (option graph): the join steps of the
  // first semi-naive round, recorded as they run, are the plan of every
  // later round
  struct GStep {
    size_t rule = 0;
    size_t t = 0;          // position in the rule's join chain (1-based)
    JoinSpec js{};         // as planned; probe columns and size come from the device
    bool last = false, filter = false;
    uint32_t head = 0;     // relation the last step appends to
    int probe_rel = -1;    // first step: the relation whose delta it probes
    uint64_t seen_probe = 0, seen_total = 0;
  };
  std::vector<GStep> grec;
  bool recording = false, grec_bad = false, graph_ready = false;
  struct GRelRes {
    uint32_t rel = 0;
    DCols F[2], D[2], fresh, alt;
    DCols ret;  // batched runs: the retired rows while the graph runs
    DBuf sort_ws, merge_ws;
    RadixPlan plan;
    bool sorted_in_alt = false;
    uint64_t Fcap = 0, Ucap = 0;
  };
  struct GStepRes {
    DBuf off, cws, wws;
    size_t wbytes = 0;
    DCols inter;
    uint64_t pcap = 0, ocap = 0;
  };
  std::vector<GRelRes> grel;
  std::vector<GStepRes> gstep;
  std::vector<uint64_t> gcap_u, gcap_i, gcap_f;  // capacities by relation / step
  DBuf gdev;
  // device-side retirement of a batched graph: RetireCtl, then the
  // relations' RetireRel, then live / conv flags and the per-instance arrays
  DBuf gret;
  uint64_t gret_room = 1;  // retired buffers start at this many times Full's capacity
  uint64_t g_retirements = 0;  // rounds whose converged rows the graph moved out of Full
  bool graph_retires() const { return opt.n_instances && opt.retire >= 0; }
  RetireCtl* g_rctl() const { return static_cast<RetireCtl*>(gret.p); }
  RetireRel* g_rrel() const {
    return reinterpret_cast<RetireRel*>(static_cast<char*>(gret.p) + 256);
  }
  cudaGraph_t ggraph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  uint64_t glaunches_per_round = 0;
  uint64_t g_rounds = 0, g_builds = 0;
  // checkpoints: the rounds a loaded checkpoint had completed, and the
  // rounds of the last cdl_run (what a checkpoint saves)
  uint64_t resume_rounds = 0, resume_iters = 0;
  std::vector<uint64_t> resume_per_round;
  uint64_t last_rounds = 0, last_iters = 0;
  std::vector<uint64_t> last_per_round;
  static constexpr uint64_t kGraphRounds = 1 << 16;  // per-round sizes the device records
  DBuf inst_last;  // batched runs: last round each instance derived a tuple
  std::vector<uint64_t> h_inst;
  std::vector<uint8_t> inst_live, inst_conv;  // rows still in full; fixpoint reached
  bool est_ready() const { return opt.estimator >= 1 && est_weights; }

  cdl_status install_weights(const float* host) {
    if (!est_w.p) est_w = alloc(sizeof(float) * kMlpParams);
    if (!est_wb.p) est_wb = alloc(sizeof(uint16_t) * kMlpParams);
    if (!est_w.p || !est_wb.p) return fail(CDL_E_NOMEM, "estimator weights");
    cudaError_t e = cudaSuccess;
    if (host)
      e = cudaMemcpyAsync(est_w.p, host, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = mlp_to_bf16(ctx, static_cast<const float*>(est_w.p), est_wb.p);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "estimator weights");
    est_weights = true;
    return CDL_OK;
  }

  // Full-batch Adam on the pinball loss, from He-uniform weights drawn by a
  // counter-based SplitMix64 stream of the seed.
  cdl_status train(const float* X, const float* y, uint64_t n, uint32_t epochs, float lr, float tau,
                   uint64_t seed, float* loss) {
    if (!X) {
      X = log_x.data();
      y = log_y.data();
      n = log_y.size();
    }
    if (n == 0 || !y) return fail(CDL_E_INVALID, "no training samples");
    std::vector<float> w(kMlpParams, 0.f);
    auto uni = [&](uint64_t i) {  // uniform in [-1, 1)
      uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return (float)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    };
    const int H = kMlpHidden, I = kMlpIn;
    const int oW2 = H * I + H, ow3 = oW2 + H * H + H;
    for (int i = 0; i < H * I; ++i) w[i] = uni(i) * std::sqrt(6.f / I);
    for (int i = 0; i < H * H; ++i) w[oW2 + i] = uni(H * I + i) * std::sqrt(6.f / H);
    for (int i = 0; i < H; ++i) w[ow3 + i] = uni(H * I + H * H + i) * std::sqrt(6.f / H);
    if (!est_w.p) est_w = alloc(sizeof(float) * kMlpParams);
    DBuf dX = alloc(sizeof(float) * I * n), dy = alloc(sizeof(float) * n),
         dout = alloc(sizeof(float) * n), ws = alloc(mlp_workspace(n)),
         g = alloc(sizeof(float) * kMlpParams), m = alloc(sizeof(float) * kMlpParams),
         v = alloc(sizeof(float) * kMlpParams);
    if (!est_w.p || !dX.p || !dy.p || !dout.p || !ws.p || !g.p || !m.p || !v.p)
      return fail(CDL_E_NOMEM, "estimator training buffers");
    float* th = static_cast<float*>(est_w.p);
    cudaError_t e = cudaMemcpyAsync(th, w.data(), sizeof(float) * kMlpParams,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dX.p, X, sizeof(float) * I * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy.p, y, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.p, 0, sizeof(float) * kMlpParams, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.p, 0, sizeof(float) * kMlpParams, st);
    for (uint32_t s = 1; s <= epochs && e == cudaSuccess; ++s) {
      e = mlp_gradient(ctx, th, static_cast<float*>(dX.p), static_cast<float*>(dy.p), n, tau,
                       static_cast<float*>(dout.p), static_cast<float*>(g.p), ws.p);
      if (e == cudaSuccess)
        e = mlp_adam(ctx, th, static_cast<float*>(g.p), static_cast<float*>(m.p),
                     static_cast<float*>(v.p), s, lr);
    }
    std::vector<float> pred(n);
    if (e == cudaSuccess)
      e = mlp_forward(ctx, th, static_cast<float*>(dX.p), n, static_cast<float*>(dout.p), ws.p);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(pred.data(), dout.p, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "estimator training");
    if (loss) {
      double l = 0;
      for (uint64_t i = 0; i < n; ++i) {
        const double r = (double)y[i] - pred[i];
        l += std::max(tau * r, (tau - 1.0) * r);
      }
      *loss = (float)(l / n);
    }
    return install_weights(nullptr);
  }

  ~cdl_engine() {
    cache.clear();
    rels.clear();
    ctl.reset();
    pool.release_all();
    hpool.release_all();
    if (h_ctl) cudaFreeHost(h_ctl);
    if (h_est) cudaFreeHost(h_est);
    if (h_batch) cudaFreeHost(h_batch);
  }

  cdl_status fail(cdl_status s, const std::string& m) {
    err = m;
    return s;
  }
  cdl_status cuda_fail(cudaError_t e, const char* where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return CDL_E_CUDA;
  }
  uint64_t* dslot(uint32_t i) { return static_cast<uint64_t*>(ctl.p) + i; }

  DBuf alloc(size_t bytes) {
    DBuf b;
    b.p = pool.get(bytes);
    if (b.p) {
      b.pool = &pool;
      b.bytes = bytes;
    }
    return b;
  }
  // k columns of cap rows in pinned host memory (the GPU accesses them in place)
  bool alloc_cols_host(DCols& d, uint32_t k, uint64_t cap) {
    d.clear();
    const size_t stride = col_stride(cap);
    d.buf.p = hpool.get(stride * k);
    if (!d.buf.p) return false;
    d.buf.pool = &hpool;
    d.buf.bytes = stride * k;
    d.k = k;
    d.cap = cap;
    for (uint32_t i = 0; i < k; ++i)
      d.c[i] = reinterpret_cast<uint32_t*>(static_cast<char*>(d.buf.p) + stride * i);
    return true;
  }
  bool alloc_cols(DCols& d, uint32_t k, uint64_t cap) {
    d.clear();
    const size_t stride = col_stride(cap);
    d.buf = alloc(stride * k);
    if (!d.buf.p) return false;
    d.k = k;
    d.cap = cap;
    for (uint32_t i = 0; i < k; ++i)
      d.c[i] = reinterpret_cast<uint32_t*>(static_cast<char*>(d.buf.p) + stride * i);
    return true;
  }

  // Copies control slots [first, first + count) and the error word to the
  // host and waits for the stream.
  cdl_status fetch(uint32_t first, uint32_t count) {
    cudaError_t e = cudaMemcpyAsync(h_ctl, dslot(kSlotErr), sizeof(uint64_t),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && count)
      e = cudaMemcpyAsync(h_ctl + first, dslot(first), sizeof(uint64_t) * count,
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "fetch");
    const uint32_t flags = (uint32_t)h_ctl[kSlotErr];
    if (flags & kErrTimeout) return fail(CDL_E_TIMEOUT, "a device-side wait ran out");
    if (flags & kErrValue) return fail(CDL_E_VALUE, "input holds the reserved value 0xFFFFFFFF");
    if (flags & kErrCapacity) return fail(CDL_E_CAPACITY, "an output buffer overflowed");
    if (flags & kErrTable) return fail(CDL_E_CAPACITY, "a hash table ran out of slots");
    return CDL_OK;
  }

  // ------------------------------------------------------------- sorting
  // Sorts d (n rows) lexicographically in place; bits[k] bounds column k.
  cdl_status sort_cols(DCols& d, const uint32_t* bits) {
    if (d.n <= 1) return CDL_OK;
    // tuner candidates: bit 0 the other digit width, bit 1 blocks of 256
    int cand = 0;
    bool measure = false;
    std::string key;
    uint32_t total = 0;
    for (uint32_t k = 0; k < d.k; ++k) total += bits[k];
    if (tuner.mode && d.n >= (1u << 14)) {
      key = "sort.k" + std::to_string(d.k) + ".b" + std::to_string(total) + ".n" +
            std::to_string(bits_of(d.n));
      cand = tuner.choose(key, 4, &measure);
    }
    const uint32_t base = digits_for(total);
    const uint32_t digit = (cand & 1) ? (base == 10 ? 8 : 10) : base;
    RadixPlan plan = make_radix_plan(d.k, bits, digit, (cand & 2) ? 256 : 512);
    if (plan.npass == 0) return CDL_OK;
    DCols alt;
    if (!alloc_cols(alt, d.k, d.n)) return fail(CDL_E_NOMEM, "sort buffer");
    DBuf ws = alloc(radix_workspace(d.n, plan.bits, plan.threads));
    if (!ws.p) return fail(CDL_E_NOMEM, "sort workspace");
    bool in_b = false;
    Tuner::Probe pr;
    if (measure) pr = tuner.start(key, cand, (double)d.n, st);
    cudaError_t e = radix_sort(ctx, plan, d.out(), alt.out(), d.n, ws.p, &in_b);
    if (e != cudaSuccess) return cuda_fail(e, "radix_sort");
    if (measure) tuner.stop(pr, st);
    if (in_b) {
      alt.n = d.n;
      std::swap(d, alt);
    }
    return CDL_OK;
  }

  // merged = full U fresh (fresh sorted, repeats allowed); delta = fresh - full.
  cdl_status merge_into(Relation& r, DCols& fresh, DCols* delta_out, uint32_t delta_slot) {
    if (r.dsm.on) return dsm_diff(r, fresh, delta_out, delta_slot);
    DCols merged, delta;
    const bool ok = r.host_full ? alloc_cols_host(merged, r.arity, r.full.n + fresh.n)
                                : alloc_cols(merged, r.arity, r.full.n + fresh.n);
    if (!ok || !alloc_cols(delta, r.arity, fresh.n)) return fail(CDL_E_NOMEM, "merge buffers");
    DBuf ws = alloc(diff_merge_workspace(r.full.n, fresh.n));
    if (!ws.p) return fail(CDL_E_NOMEM, "merge workspace");
    cudaError_t e = diff_merge(ctx, r.arity, r.full.in(), r.full.n, fresh.in(), fresh.n,
                               delta.out(), merged.out(), dslot(delta_slot), ws.p);
    if (e != cudaSuccess) return cuda_fail(e, "diff_merge");
    merged.n = r.full.n;  // grows by |delta| once it is read back
    r.full = std::move(merged);
    r.version[kFull]++;
    r.delta_version = r.version[kFull];
    if (delta_out) *delta_out = std::move(delta);
    return CDL_OK;
  }

  // ------------------------------------------- Algorithm 2 (option dedup)
  // Derived relations whose Full no rule variant reads after round 1 (every
  // rule that names them has no other derived body atom, so its semi-naive
  // variant reads their delta only) keep Full in the decomposed form.
  void dsm_select() {
    std::vector<uint8_t> full_read(rels.size(), 0);
    for (const RuleR& r : rules) {
      uint32_t nidb = 0;
      for (const AtomR& a : r.body) nidb += rels[a.rel]->idb ? 1u : 0u;
      if (nidb >= 2)
        for (const AtomR& a : r.body)
          if (rels[a.rel]->idb) full_read[a.rel] = 1;
    }
    for (size_t i = 0; i < rels.size(); ++i) {
      Relation& R = *rels[i];
      R.dsm.reset();
      R.dsm.on = opt.dedup > 0 && R.idb && !full_read[i] && !opt.n_instances;
      // out of core: Full that only step (d) reads lives in pinned host memory
      R.host_full = opt.host_full > 0 && R.idb && !full_read[i] && !opt.n_instances && !R.dsm.on;
    }
  }

  DsmView dsm_view(const Relation& R) const {
    DsmView v;
    v.raw = R.dsm.raw.in();
    v.n = R.dsm.raw.n;
    for (uint32_t k = 0; k < R.arity; ++k) {
      v.ids[k] = R.dsm.idx[k].c[1];
      v.table[k] = static_cast<const Slot*>(R.dsm.table[k].p);
      v.mask[k] = R.dsm.slots[k] ? R.dsm.slots[k] - 1 : 0;
    }
    v.mm = static_cast<const uint2*>(R.dsm.mm.p);
    v.mm_mask = R.dsm.mm_slots ? R.dsm.mm_slots - 1 : 0;
    return v;
  }

  // The unique hashmap of every column over its sorted index.
  cdl_status dsm_tables(Relation& R) {
    Dsm& D = R.dsm;
    for (uint32_t k = 0; k < R.arity; ++k) {
      uint64_t distinct = 0;
      if (D.raw.n) {
        cudaError_t e = count_heads(ctx, D.idx[k].c[0], nullptr, D.raw.n, dslot(kSlotScratch));
        if (e != cudaSuccess) return cuda_fail(e, "count_heads");
        cdl_status r = fetch(kSlotScratch, 1);
        if (r != CDL_OK) return r;
        distinct = h_ctl[kSlotScratch];
      }
      const uint64_t slots = table_slots(distinct, hash_load);
      if (slots != D.slots[k] || !D.table[k].p) {
        D.table[k] = alloc(slots * sizeof(Slot));
        if (!D.table[k].p) return fail(CDL_E_NOMEM, "decomposed hashmap");
        D.slots[k] = slots;
      }
      cudaError_t e = hash_build(ctx, D.idx[k].c[0], nullptr, D.raw.n,
                                 static_cast<Slot*>(D.table[k].p), slots);
      if (e != cudaSuccess) return cuda_fail(e, "hash_build");
    }
    return CDL_OK;
  }

  // Multimap of column 0 sized for cap rows at load 0.5, holding rows [0, n).
  cdl_status dsm_multimap(Relation& R, uint64_t cap) {
    Dsm& D = R.dsm;
    D.mm_slots = table_slots(cap, 0.5);
    D.mm = alloc(D.mm_slots * 8);
    if (!D.mm.p) return fail(CDL_E_NOMEM, "decomposed multimap");
    cudaError_t e = cudaMemsetAsync(D.mm.p, 0xFF, D.mm_slots * 8, st);
    if (e == cudaSuccess)
      e = mm_insert(ctx, D.raw.c[0], D.raw.n, 0, static_cast<uint2*>(D.mm.p), D.mm_slots);
    return e == cudaSuccess ? CDL_OK : cuda_fail(e, "multimap");
  }

  // Column k's (value, id) entries of rows [first, first + n) of src, in
  // (value, id) order: src is sorted with column 0 first, so column 0's
  // entries already are; the others sort by value, stably (ids ascend).
  cdl_status dsm_entries(const Relation& R, const DCols& src, uint32_t k, uint64_t first,
                         DCols& out) {
    const uint64_t n = src.n;
    if (!alloc_cols(out, 2, n)) return fail(CDL_E_NOMEM, "index entries");
    out.n = n;
    cudaError_t e = n ? cudaMemcpyAsync(out.c[0], src.c[k], n * 4, cudaMemcpyDeviceToDevice, st)
                      : cudaSuccess;
    if (e == cudaSuccess) e = iota_u32(ctx, out.c[1], n, (uint32_t)first);
    if (e != cudaSuccess) return cuda_fail(e, "index entries");
    if (k == 0 || n <= 1) return CDL_OK;
    const uint32_t bits[2] = {bits_of(R.bound[k]), 0};  // by value only: a stable pass keeps ids ascending
    return sort_cols(out, bits);
  }

  // Full, as loaded or left by round 1, becomes the decomposed form.
  cdl_status dsm_build(Relation& R) {
    Dsm& D = R.dsm;
    const uint64_t n0 = R.full.n;
    if (!alloc_cols(D.raw, R.arity, std::max<uint64_t>(2 * n0, 1 << 16)))
      return fail(CDL_E_NOMEM, "decomposed rows");
    for (uint32_t k = 0; k < R.arity && n0; ++k) {
      cudaError_t e = cudaMemcpyAsync(D.raw.c[k], R.full.c[k], n0 * 4, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "decomposed rows");
    }
    D.raw.n = n0;
    cdl_status r = CDL_OK;
    if (opt.dedup == 1) {
      for (uint32_t k = 0; k < R.arity && r == CDL_OK; ++k) r = dsm_entries(R, R.full, k, 0, D.idx[k]);
      if (r == CDL_OK) r = dsm_tables(R);
    } else {
      r = dsm_multimap(R, D.raw.cap);
    }
    if (r != CDL_OK) return r;
    R.full.clear();  // the rows live in the decomposed form until the run ends
    R.full.k = R.arity;
    R.full.n = n0;
    D.init = true;
    return CDL_OK;
  }

  // Step (d) by Algorithm 2: delta = the sorted fresh rows that repeat
  // neither their predecessor nor a row of Full; |delta| into delta_slot.
  cdl_status dsm_diff(Relation& R, DCols& fresh, DCols* delta_out, uint32_t delta_slot) {
    if (!R.dsm.init) {
      cdl_status r = dsm_build(R);
      if (r != CDL_OK) return r;
    }
    const uint64_t n = fresh.n;
    DBuf flags = alloc(4 * (n ? n : 1)), off = alloc(8 * (n ? n : 1)), ws = alloc(scan_workspace(n));
    DCols delta;
    if (!flags.p || !off.p || !ws.p || !alloc_cols(delta, R.arity, n))
      return fail(CDL_E_NOMEM, "dedup buffers");
    const DsmView v = dsm_view(R);
    uint32_t* f = static_cast<uint32_t*>(flags.p);
    uint64_t* o = static_cast<uint64_t*>(off.p);
    cudaError_t e = dsm_probe(ctx, R.arity, fresh.in(), n, v, opt.dedup == 2, f);
    if (e == cudaSuccess) e = exclusive_scan(ctx, f, n, o, dslot(delta_slot), ws.p);
    if (e == cudaSuccess) e = compact_rows(ctx, R.arity, fresh.in(), n, f, o, delta.out());
    if (e != cudaSuccess) return cuda_fail(e, "dedup");
    R.version[kFull]++;
    if (delta_out) *delta_out = std::move(delta);
    return CDL_OK;
  }

  // The union, once |delta| is known: delta appended to the rows (new ids
  // n0 ..), its entries merged into every column's sorted index, the
  // hashmaps rebuilt (or delta's column 0 added to the multimap).
  cdl_status dsm_append(Relation& R) {
    Dsm& D = R.dsm;
    const uint64_t n0 = D.raw.n, nd = R.delta.n, n1 = n0 + nd;
    if (nd == 0) return CDL_OK;
    if (n1 > D.raw.cap) {
      DCols grown;
      if (!alloc_cols(grown, R.arity, std::max<uint64_t>(2 * n1, D.raw.cap * 2)))
        return fail(CDL_E_NOMEM, "decomposed rows");
      for (uint32_t k = 0; k < R.arity; ++k) {
        cudaError_t e = cudaMemcpyAsync(grown.c[k], D.raw.c[k], n0 * 4, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "decomposed rows");
      }
      D.raw = std::move(grown);
    }
    for (uint32_t k = 0; k < R.arity; ++k) {
      cudaError_t e = cudaMemcpyAsync(D.raw.c[k] + n0, R.delta.c[k], nd * 4,
                                      cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "decomposed rows");
    }
    D.raw.n = n1;
    if (opt.dedup == 2) {
      if (n1 > D.mm_slots / 2) return dsm_multimap(R, D.raw.cap);
      cudaError_t e = mm_insert(ctx, R.delta.c[0], nd, (uint32_t)n0, static_cast<uint2*>(D.mm.p),
                                D.mm_slots);
      return e == cudaSuccess ? CDL_OK : cuda_fail(e, "multimap");
    }
    for (uint32_t k = 0; k < R.arity; ++k) {
      DCols add, merged, unused;
      cdl_status r = dsm_entries(R, R.delta, k, n0, add);
      if (r != CDL_OK) return r;
      if (!alloc_cols(merged, 2, n1) || !alloc_cols(unused, 2, nd))
        return fail(CDL_E_NOMEM, "index merge");
      DBuf ws = alloc(diff_merge_workspace(n0, nd));
      if (!ws.p) return fail(CDL_E_NOMEM, "index merge");
      // ids are distinct, so no entry repeats: the merge keeps them all
      cudaError_t e = diff_merge(ctx, 2, D.idx[k].in(), n0, add.in(), nd, unused.out(),
                                 merged.out(), dslot(kSlotScratch), ws.p);
      if (e != cudaSuccess) return cuda_fail(e, "index merge");
      merged.n = n1;
      D.idx[k] = std::move(merged);
    }
    return dsm_tables(R);
  }

  // At the end of the run Full goes back to sorted rows (what export and
  // checkpoints read): the rows sorted lexicographically.
  cdl_status dsm_finish() {
    for (auto& rp : rels) {
      Relation& R = *rp;
      if (!R.dsm.on || !R.dsm.init) continue;
      DCols rows;
      const uint64_t n = R.dsm.raw.n;
      if (!alloc_cols(rows, R.arity, n)) return fail(CDL_E_NOMEM, "sorted rows");
      for (uint32_t k = 0; k < R.arity && n; ++k) {
        cudaError_t e = cudaMemcpyAsync(rows.c[k], R.dsm.raw.c[k], n * 4, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "sorted rows");
      }
      rows.n = n;
      uint32_t bits[kMaxK];
      for (uint32_t k = 0; k < R.arity; ++k) bits[k] = bits_of(R.bound[k]);
      cdl_status r = sort_cols(rows, bits);
      if (r != CDL_OK) return r;
      R.full = std::move(rows);
      R.version[kFull]++;
      R.dsm.reset();
      R.dsm.on = true;  // stays marked: the run used the decomposed form
    }
    return CDL_OK;
  }

  // ------------------------------------------------------------- indexes
  cdl_status get_index(const Src& s, const std::vector<uint32_t>& key, Index** out,
                       std::unique_ptr<Index>& temp) {
    const bool cacheable = s.rel >= 0;
    if (cacheable) {
      const uint64_t v = rels[s.rel]->version[s.ver];
      for (auto& ix : cache)
        if (ix->rel == s.rel && ix->ver == s.ver && ix->version == v && ix->key == key) {
          *out = ix.get();
          return CDL_OK;
        }
    }
    auto ix = std::make_unique<Index>();
    ix->rel = s.rel;
    ix->ver = s.ver;
    ix->version = cacheable ? rels[s.rel]->version[s.ver] : 0;
    ix->key = key;
    ix->n = s.n;
    bool prefix = true;
    for (size_t i = 0; i < key.size(); ++i) prefix &= key[i] == i;
    if (prefix) {
      for (uint32_t c = 0; c < s.k; ++c) ix->cols[c] = s.c[c];
    } else {
      std::vector<uint32_t> perm = key;
      for (uint32_t c = 0; c < s.k; ++c)
        if (std::find(key.begin(), key.end(), c) == key.end()) perm.push_back(c);
      uint32_t pbits[kMaxK];
      for (uint32_t i = 0; i < s.k; ++i) pbits[i] = s.bits[perm[i]];
      Index* prev = nullptr;
      if (cacheable && s.ver == kFull) {
        const Relation& R = *rels[s.rel];
        for (auto& p : prev_full)
          if (p->rel == s.rel && p->key == key && p->version + 1 == R.version[kFull] &&
              R.delta_version == R.version[kFull] && p->n + R.delta.n == s.n)
            prev = p.get();
      }
      if (prev) {  // previous version's sorted copy merged with the round's delta
        const Relation& R = *rels[s.rel];
        const uint64_t nd = R.delta.n;
        DCols dp, unused;
        if (!alloc_cols(dp, s.k, nd) || !alloc_cols(unused, s.k, nd) ||
            !alloc_cols(ix->sorted, s.k, s.n))
          return fail(CDL_E_NOMEM, "index merge");
        dp.n = nd;
        for (uint32_t i = 0; i < s.k && nd; ++i) {
          cudaError_t e = cudaMemcpyAsync(dp.c[i], R.delta.c[perm[i]], nd * 4,
                                          cudaMemcpyDeviceToDevice, st);
          if (e != cudaSuccess) return cuda_fail(e, "index merge");
        }
        cdl_status r = sort_cols(dp, pbits);
        if (r != CDL_OK) return r;
        DBuf ws = alloc(diff_merge_workspace(prev->n, nd));
        if (!ws.p) return fail(CDL_E_NOMEM, "index merge");
        // delta and the previous Full share no tuple: the merge keeps them all
        cudaError_t e = diff_merge(ctx, s.k, prev->sorted.in(), prev->n, dp.in(), nd,
                                   unused.out(), ix->sorted.out(), dslot(kSlotScratch), ws.p);
        if (e != cudaSuccess) return cuda_fail(e, "index merge");
        ix->sorted.n = s.n;
        ++index_merges;
        prev_full.erase(std::remove_if(prev_full.begin(), prev_full.end(),
                                       [&](const std::unique_ptr<Index>& p) { return p.get() == prev; }),
                        prev_full.end());
      } else {
        if (!alloc_cols(ix->sorted, s.k, s.n)) return fail(CDL_E_NOMEM, "index copy");
        ix->sorted.n = s.n;
        for (uint32_t i = 0; i < s.k; ++i) {
          cudaError_t e = cudaMemcpyAsync(ix->sorted.c[i], s.c[perm[i]], s.n * 4,
                                          cudaMemcpyDeviceToDevice, st);
          if (e != cudaSuccess) return cuda_fail(e, "index copy");
        }
        cdl_status r = sort_cols(ix->sorted, pbits);
        if (r != CDL_OK) return r;
      }
      for (uint32_t i = 0; i < s.k; ++i) ix->cols[perm[i]] = ix->sorted.c[i];
    }
    const uint32_t* k0 = ix->cols[key[0]];
    const uint32_t* k1 = key.size() > 1 ? ix->cols[key[1]] : nullptr;
    cudaError_t e = count_heads(ctx, k0, k1, s.n, dslot(kSlotScratch));
    if (e != cudaSuccess) return cuda_fail(e, "count_heads");
    cdl_status r = fetch(kSlotScratch, 1);
    if (r != CDL_OK) return r;
    ix->distinct = h_ctl[kSlotScratch];
    double load = hash_load;
    if (tuner.mode && ix->distinct >= 4096) {  // candidates: the configured load, 0.6, 0.7, 0.8
      static const double kLoads[4] = {0.0, 0.6, 0.7, 0.8};
      bool unused;
      ix->tkey = "load.n" + std::to_string(bits_of(ix->distinct));
      ix->tcand = tuner.choose(ix->tkey, 4, &unused);
      if (ix->tcand) load = kLoads[ix->tcand];
    }
    ix->slots = table_slots(ix->distinct, load);
    ix->table = alloc(ix->slots * sizeof(Slot));
    if (!ix->table.p) return fail(CDL_E_NOMEM, "hash table");
    e = hash_build(ctx, k0, k1, s.n, static_cast<Slot*>(ix->table.p), ix->slots);
    if (e != cudaSuccess) return cuda_fail(e, "hash_build");
    *out = ix.get();
    if (cacheable)
      cache.push_back(std::move(ix));
    else
      temp = std::move(ix);
    return CDL_OK;
  }

  void evict_stale() {
    // a Full index one version behind, sorted by non-leading columns, waits
    // for the next version's index (at most one per relation and key)
    prev_full.erase(std::remove_if(prev_full.begin(), prev_full.end(),
                                   [&](const std::unique_ptr<Index>& p) {
                                     return p->version + 1 < rels[p->rel]->version[kFull];
                                   }),
                    prev_full.end());
    for (auto& ix : cache) {
      const Relation& R = *rels[ix->rel];
      if (ix->version == R.version[ix->ver] || ix->ver != kFull || !ix->sorted.buf.p ||
          ix->version + 1 != R.version[kFull])
        continue;
      prev_full.erase(std::remove_if(prev_full.begin(), prev_full.end(),
                                     [&](const std::unique_ptr<Index>& p) {
                                       return p->rel == ix->rel && p->key == ix->key;
                                     }),
                      prev_full.end());
      ix->table.reset();  // only the sorted copy is merged
      prev_full.push_back(std::move(ix));
    }
    cache.erase(std::remove_if(cache.begin(), cache.end(),
                               [&](const std::unique_ptr<Index>& ix) {
                                 return !ix || ix->version != rels[ix->rel]->version[ix->ver];
                               }),
                cache.end());
  }

  // --------------------------------------------------------- fresh buffers
  cdl_status ensure_fresh(Relation& r, uint64_t extra) {
    const uint64_t need = r.fresh_ub + extra;
    // a round's new rows are sorted and merged with 32-bit row counts: the
    // exact count of a join (or a bound on it) past that stops the run
    // before anything is allocated or written
    if (need > 0xFFFFFFFFull)
      return fail(CDL_E_CAPACITY, "relation " + r.name + " would receive more than 2^32 new "
                                  "tuples in one round");
    if (need <= r.fresh.cap && r.fresh.buf.p) {
      r.fresh_ub = need;
      return CDL_OK;
    }
    DCols nf;
    uint64_t cap = std::max<uint64_t>(need, r.fresh.cap + r.fresh.cap / 2);
    if (cap < 1024) cap = 1024;
    if (!alloc_cols(nf, r.arity, cap)) return fail(CDL_E_NOMEM, "new-tuple buffer");
    // rows past the old capacity were never written (a claim beyond the
    // buffer marks the relation for an exact redo): copy only what exists
    const uint64_t rows = std::min(r.fresh_ub, r.fresh.cap);
    if (r.fresh.buf.p && rows) {
      for (uint32_t k = 0; k < r.arity; ++k) {
        cudaError_t e = cudaMemcpyAsync(nf.c[k], r.fresh.c[k], rows * 4,
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "grow new-tuple buffer");
      }
    }
    r.fresh = std::move(nf);
    r.fresh_ub = need;
    return CDL_OK;
  }

  // ------------------------------------------------------------- atoms
  Src rel_src(uint32_t rel, int ver) {
    Relation& R = *rels[rel];
    const DCols& d = ver == kDelta ? R.delta : R.full;
    Src s;
    for (uint32_t k = 0; k < R.arity; ++k) {
      s.c[k] = d.c[k];
      s.bits.push_back(bits_of(R.bound[k]));
    }
    s.n = d.n;
    s.k = R.arity;
    s.rel = (int)rel;
    s.ver = ver;
    return s;
  }

  // The atom's relation version as a table over its distinct variables,
  // through a selection when it holds constants or repeated variables.
  cdl_status atom_src(const AtomR& a, int ver, Src& out) {
    Src base = rel_src(a.rel, ver);
    std::vector<uint32_t> vars;
    bool plain = true;
    for (const Term& t : a.t) {
      if (t.is_const || std::find(vars.begin(), vars.end(), t.v) != vars.end())
        plain = false;
      else
        vars.push_back(t.v);
    }
    if (plain) {
      out = std::move(base);
      out.vars = vars;
      return CDL_OK;
    }
    SelectSpec sp{};
    sp.in = base.in();
    sp.in_k = base.k;
    sp.n = base.n;
    std::vector<uint32_t> first_col;
    std::vector<uint32_t> seen;
    for (uint32_t k = 0; k < a.t.size(); ++k) {
      const Term& t = a.t[k];
      if (t.is_const) {
        sp.const_col[sp.n_const] = k;
        sp.const_val[sp.n_const++] = t.v;
      } else {
        auto it = std::find(seen.begin(), seen.end(), t.v);
        if (it != seen.end()) {
          sp.same[sp.n_same][0] = first_col[it - seen.begin()];
          sp.same[sp.n_same++][1] = k;
        } else {
          seen.push_back(t.v);
          first_col.push_back(k);
        }
      }
    }
    sp.out_k = (uint32_t)seen.size();
    for (uint32_t i = 0; i < sp.out_k; ++i) sp.out[i] = Ref{0, first_col[i]};
    out = Src();
    out.vars = seen;
    out.k = sp.out_k;
    if (sp.out_k == 0) {  // an atom without variables only tests for a matching tuple
      sp.out_k = 1;
      sp.out[0] = Ref{0, 0};
    }
    if (!alloc_cols(out.owned, sp.out_k, base.n)) return fail(CDL_E_NOMEM, "selection buffer");
    for (uint32_t i = 0; i < out.k; ++i) {
      out.c[i] = out.owned.c[i];
      out.bits.push_back(base.bits[first_col[i]]);
    }
    cudaError_t e = cudaMemsetAsync(dslot(kSlotAux), 0, 8, st);
    if (e == cudaSuccess) e = select_project(ctx, sp, out.owned.out(), dslot(kSlotAux), base.n);
    if (e != cudaSuccess) return cuda_fail(e, "select");
    cdl_status r = fetch(kSlotAux, 1);
    if (r != CDL_OK) return r;
    out.n = out.owned.n = h_ctl[kSlotAux];
    return CDL_OK;
  }

  // --------------------------------------------------------------- rules
  cdl_status eval_copy(const RuleR& rule, int ver) {
    if (recording) grec_bad = true;
    const AtomR& a = rule.body[0];
    Src base = rel_src(a.rel, ver);
    if (base.n == 0) return CDL_OK;
    SelectSpec sp{};
    sp.in = base.in();
    sp.in_k = base.k;
    sp.n = base.n;
    std::map<uint32_t, uint32_t> col_of;
    for (uint32_t k = 0; k < a.t.size(); ++k) {
      const Term& t = a.t[k];
      if (t.is_const) {
        sp.const_col[sp.n_const] = k;
        sp.const_val[sp.n_const++] = t.v;
      } else if (col_of.count(t.v)) {
        sp.same[sp.n_same][0] = col_of[t.v];
        sp.same[sp.n_same++][1] = k;
      } else {
        col_of[t.v] = k;
      }
    }
    sp.out_k = (uint32_t)rule.head.t.size();
    for (uint32_t k = 0; k < sp.out_k; ++k) {
      const Term& t = rule.head.t[k];
      sp.out[k] = t.is_const ? Ref{2, t.v} : Ref{0, col_of.at(t.v)};
    }
    for (auto& ne : rule.neq) {
      sp.neq[sp.n_neq][0] = Ref{0, col_of.at(ne.first)};
      sp.neq[sp.n_neq++][1] = Ref{0, col_of.at(ne.second)};
    }
    Relation& H = *rels[rule.head.rel];
    cdl_status r = ensure_fresh(H, base.n);
    if (r != CDL_OK) return r;
    cudaError_t e = select_project(ctx, sp, H.fresh.out(), dslot(kSlotCursor + rule.head.rel),
                                   H.fresh.cap, soft_overflow());
    return e == cudaSuccess ? CDL_OK : cuda_fail(e, "copy rule");
  }

  // One variant of a rule with >= 2 body atoms: a left-deep chain of
  // hash joins starting at atom `start` (the delta atom of the variant).
  // Writes the head tuples of a rule whose join chain is a single table
  // (s) or empty (s == null: a body of variable-free atoms, all matched).
  cdl_status emit_from(const RuleR& rule, const Src* s, const Src& any) {
    if (recording) grec_bad = true;
    SelectSpec sp{};
    if (s) {
      sp.in = s->in();
      sp.in_k = s->k;
      sp.n = s->n;
    } else {
      sp.in.c[0] = any.owned.c[0];
      sp.in_k = 1;
      sp.n = 1;
    }
    auto col = [&](uint32_t v) {
      return (uint32_t)(std::find(s->vars.begin(), s->vars.end(), v) - s->vars.begin());
    };
    sp.out_k = (uint32_t)rule.head.t.size();
    for (uint32_t k = 0; k < sp.out_k; ++k) {
      const Term& t = rule.head.t[k];
      sp.out[k] = t.is_const ? Ref{2, t.v} : Ref{0, col(t.v)};
    }
    for (auto& ne : rule.neq) {
      sp.neq[sp.n_neq][0] = Ref{0, col(ne.first)};
      sp.neq[sp.n_neq++][1] = Ref{0, col(ne.second)};
    }
    Relation& H = *rels[rule.head.rel];
    cdl_status r = ensure_fresh(H, sp.n);
    if (r != CDL_OK) return r;
    cudaError_t e = select_project(ctx, sp, H.fresh.out(), dslot(kSlotCursor + rule.head.rel),
                                   H.fresh.cap, soft_overflow());
    return e == cudaSuccess ? CDL_OK : cuda_fail(e, "project");
  }

  // One variant of a rule with >= 2 body atoms: a left-deep chain of
  // hash joins starting at atom `start` (the delta atom of the variant).
  // Variable-free atoms only gate the rule; atoms that share no variable
  // with the chain so far join as a cross product.
  // The index of a relation version on key columns is cached.
  bool index_cached(const Src& B, const std::vector<uint32_t>& key) const {
    if (B.rel < 0) return false;
    const uint64_t v = rels[B.rel]->version[B.ver];
    for (auto& ix : cache)
      if (ix && ix->rel == B.rel && ix->ver == B.ver && ix->version == v && ix->key == key)
        return true;
    return false;
  }
  // The previous Full version's index on key waits to be merged with delta.
  bool index_incremental(const Src& B, const std::vector<uint32_t>& key) const {
    if (B.rel < 0 || B.ver != kFull) return false;
    const Relation& R = *rels[B.rel];
    for (auto& p : prev_full)
      if (p->rel == B.rel && p->key == key && p->version + 1 == R.version[kFull] &&
          R.delta_version == R.version[kFull])
        return true;
    return false;
  }
  // Bytes a first join moves with B as its build side and P probing it:
  // B's index (nothing when cached or when B is an input relation, whose
  // index is built once for the run; otherwise the distinct-key count and
  // the hash build, plus, for a key that is not B's leading columns, the
  // previous version's sorted copy merged with delta where that exists or
  // a copy sorted in about five radix passes; a derived relation's Full is
  // priced at the merge, which it reaches from its second round) and the
  // probe side's count and write passes (24 + 36 bytes per probe row).  The
  // output is the same either way.
  double orient_bytes(const Src& B, const Src& P) const {
    std::vector<uint32_t> key;
    for (uint32_t bc = 0; bc < B.vars.size() && key.size() < 2; ++bc)
      if (std::find(P.vars.begin(), P.vars.end(), B.vars[bc]) != P.vars.end()) key.push_back(bc);
    const double n = (double)B.n, k = (double)B.k;
    // a launch (or a host wait) priced as the bytes HBM moves meanwhile, ~3 us
    const double kLaunch = opt.plan_launch_bytes > 0.0 ? opt.plan_launch_bytes : 2e7;
    double idx = 0.0;
    // an input relation's index is built once and kept for the whole run
    const bool static_rel = B.rel >= 0 && !rels[B.rel]->idb;
    if (!key.empty() && !static_rel && !index_cached(B, key)) {
      bool prefix = true;
      for (size_t i = 0; i < key.size(); ++i) prefix &= key[i] == i;
      // distinct-key count (with its read-back) and hash build: ~8 launches
      idx = 8.0 * n * (double)key.size() + 4.0 * n + 8.0 * kLaunch;
      // a derived relation's Full is sorted once, then merged with each
      // round's delta: priced at that steady rate
      const bool kept = index_incremental(B, key) ||
                        (B.rel >= 0 && B.ver == kFull && rels[B.rel]->idb);
      if (!prefix) idx += (kept ? 8.0 * k * n : 4.0 * k * n * 12.0) + 16.0 * kLaunch;
    }
    return idx + 60.0 * (double)P.n;
  }

  // Key columns of atom C probed from P beside a join of P with B (a star
  // join): every variable C shares with P or B is one of P's, one or two of
  // them (ckey: C's columns, cpkey: P's), and B shares a variable with P.
  static bool star_keys(const Src& P, const Src& B, const Src& C, std::vector<uint32_t>& ckey,
                        std::vector<uint32_t>& cpkey) {
    ckey.clear();
    cpkey.clear();
    bool shared = false;
    for (uint32_t v : B.vars) shared |= std::find(P.vars.begin(), P.vars.end(), v) != P.vars.end();
    if (!shared) return false;
    for (uint32_t cc = 0; cc < C.vars.size(); ++cc) {
      auto it = std::find(P.vars.begin(), P.vars.end(), C.vars[cc]);
      if (it != P.vars.end()) {
        ckey.push_back(cc);
        cpkey.push_back((uint32_t)(it - P.vars.begin()));
      } else if (std::find(B.vars.begin(), B.vars.end(), C.vars[cc]) != B.vars.end()) {
        return false;
      }
    }
    return !ckey.empty() && ckey.size() <= 2;
  }

  cdl_status eval_join(const RuleR& rule, const std::vector<int>& vers, size_t start) {
    const size_t nb_all = rule.body.size();
    std::vector<Src> atoms(nb_all);
    std::vector<size_t> chain;
    for (size_t i = 0; i < nb_all; ++i) {
      cdl_status r = atom_src(rule.body[i], vers[i], atoms[i]);
      if (r != CDL_OK) return r;
      if (atoms[i].n == 0) return CDL_OK;  // joins with an empty table derive nothing
      if (!atoms[i].vars.empty()) chain.push_back(i);
    }
    if (chain.size() <= 1) {
      if (est_plan) return CDL_OK;
      return emit_from(rule, chain.empty() ? nullptr : &atoms[chain[0]], atoms[0]);
    }
    if (std::find(chain.begin(), chain.end(), start) == chain.end()) start = chain[0];
    const size_t nb = chain.size();
    std::vector<size_t> order{start};
    std::vector<uint32_t> bound = atoms[start].vars;
    std::vector<bool> used(nb_all, true);
    for (size_t i : chain) used[i] = false;
    used[start] = true;
    for (size_t t = 1; t < nb; ++t) {
      size_t pick = nb_all;
      for (size_t i : chain) {
        if (used[i]) continue;
        for (uint32_t v : atoms[i].vars)
          if (std::find(bound.begin(), bound.end(), v) != bound.end()) {
            pick = i;
            break;
          }
        if (pick != nb_all) break;
      }
      if (pick == nb_all)  // nothing shares a variable: cross product with the next atom
        for (size_t i : chain)
          if (!used[i]) {
            pick = i;
            break;
          }
      used[pick] = true;
      order.push_back(pick);
      for (uint32_t v : atoms[pick].vars)
        if (std::find(bound.begin(), bound.end(), v) == bound.end()) bound.push_back(v);
    }
    std::vector<bool> neq_done(rule.neq.size(), false);
    Src left = std::move(atoms[start]);
    for (size_t t = 1; t < nb; ++t) {
      Src& right = atoms[order[t]];
      bool last = t + 1 == nb;
      // the chain's last atom, where it may join this step as a star
      Src* const after = !last && t + 2 == nb && opt.star >= 0 && !est_plan
                             ? &atoms[order[t + 1]] : nullptr;
      std::vector<uint32_t> ckey, cpkey;
      // roles: the first join may build on either atom; later joins build on the atom
      bool build_right = true;
      if (t == 1) {
        const bool right_static = right.rel >= 0 && !rels[right.rel]->idb;
        const bool left_static = left.rel >= 0 && !rels[left.rel]->idb;
        if (!right_static && (left_static || left.n < right.n)) build_right = false;
        // the learned form: the orientation that moves fewer bytes (a star
        // join, which writes no intermediate table, is kept where it applies)
        if (opt.estimator >= 1 && !recording && !left.vars.empty() && !right.vars.empty() &&
            !(build_right && after && star_keys(left, right, *after, ckey, cpkey)))
          build_right = orient_bytes(right, left) <= orient_bytes(left, right);
      }
      Src& P = build_right ? left : right;
      Src& B = build_right ? right : left;
      // a star join: the last atom keys on the probe side's variables alone,
      // so both build sides are probed from each probe row and the table
      // between the two joins is never written
      Src* const C = after && build_right && star_keys(P, B, *after, ckey, cpkey) ? after : nullptr;
      if (C) last = true;
      std::vector<uint32_t> pkey, bkey;
      for (uint32_t bc = 0; bc < B.vars.size(); ++bc) {
        auto it = std::find(P.vars.begin(), P.vars.end(), B.vars[bc]);
        if (it != P.vars.end()) {
          bkey.push_back(bc);
          pkey.push_back((uint32_t)(it - P.vars.begin()));
        }
      }
      auto ref_of = [&](uint32_t v) -> Ref {
        auto it = std::find(P.vars.begin(), P.vars.end(), v);
        if (it != P.vars.end()) return Ref{0, (uint32_t)(it - P.vars.begin())};
        it = std::find(B.vars.begin(), B.vars.end(), v);
        if (it != B.vars.end() || !C) return Ref{1, (uint32_t)(it - B.vars.begin())};
        it = std::find(C->vars.begin(), C->vars.end(), v);
        return Ref{3, (uint32_t)(it - C->vars.begin())};
      };
      auto avail = [&](uint32_t v) {
        return std::find(P.vars.begin(), P.vars.end(), v) != P.vars.end() ||
               std::find(B.vars.begin(), B.vars.end(), v) != B.vars.end() ||
               (C && std::find(C->vars.begin(), C->vars.end(), v) != C->vars.end());
      };
      std::vector<uint32_t> hkey(bkey.begin(), bkey.begin() + std::min<size_t>(2, bkey.size()));
      JoinSpec js{};
      js.probe = P.in();
      js.n_probe = P.n;
      std::unique_ptr<Index> temp_ix;
      Index* ix = nullptr;
      cdl_status r = CDL_OK;
      if (hkey.empty()) {
        if (B.n > 0xFFFFFFFFull) return fail(CDL_E_CAPACITY, "cross product side too large");
        js.cross = 1;
        js.n_build = (uint32_t)B.n;
        js.pk0 = 0;
        js.pk1 = 0xFFu;
        for (uint32_t c = 0; c < B.k; ++c) js.build.c[c] = B.c[c];
        js.slots = 1;
      } else {
        r = get_index(B, hkey, &ix, temp_ix);
        if (r != CDL_OK) return r;
        js.pk0 = pkey[0];
        js.pk1 = pkey.size() > 1 ? pkey[1] : 0xFFu;
        for (uint32_t c = 0; c < B.k; ++c) js.build.c[c] = ix->cols[c];
        js.table = static_cast<const Slot*>(ix->table.p);
        js.slots = ix->slots;
      }
      std::unique_ptr<Index> temp_ix2;
      Index* ix2 = nullptr;
      if (C) {
        r = get_index(*C, ckey, &ix2, temp_ix2);
        if (r != CDL_OK) return r;
        js.star = 1;
        js.qk0 = cpkey[0];
        js.qk1 = cpkey.size() > 1 ? cpkey[1] : 0xFFu;
        for (uint32_t c = 0; c < C->k; ++c) js.build2.c[c] = ix2->cols[c];
        js.table2 = static_cast<const Slot*>(ix2->table.p);
        js.slots2 = ix2->slots;
        ++star_joins;
      }
      for (size_t q = 2; q < bkey.size(); ++q) {
        if (js.n_eq >= 4) return fail(CDL_E_INVALID, "too many shared variables");
        js.eq[js.n_eq][0] = Ref{0, pkey[q]};
        js.eq[js.n_eq++][1] = Ref{1, bkey[q]};
      }
      for (size_t q = 0; q < rule.neq.size(); ++q) {
        if (neq_done[q] || !avail(rule.neq[q].first) || !avail(rule.neq[q].second)) continue;
        if (js.n_neq >= 4) return fail(CDL_E_INVALID, "too many inequalities");
        js.neq[js.n_neq][0] = ref_of(rule.neq[q].first);
        js.neq[js.n_neq++][1] = ref_of(rule.neq[q].second);
        neq_done[q] = true;
      }
      Src next;
      if (last) {
        js.out_k = (uint32_t)rule.head.t.size();
        for (uint32_t k = 0; k < js.out_k; ++k) {
          const Term& tm = rule.head.t[k];
          js.out[k] = tm.is_const ? Ref{2, tm.v} : ref_of(tm.v);
        }
      } else {
        std::vector<uint32_t> need;
        for (const Term& tm : rule.head.t)
          if (!tm.is_const) need.push_back(tm.v);
        for (size_t q = 0; q < rule.neq.size(); ++q)
          if (!neq_done[q]) {
            need.push_back(rule.neq[q].first);
            need.push_back(rule.neq[q].second);
          }
        for (size_t u = t + 1; u < nb; ++u)
          for (uint32_t v : atoms[order[u]].vars) need.push_back(v);
        for (const std::vector<uint32_t>* vs : {&P.vars, &B.vars})
          for (uint32_t v : *vs)
            if (std::find(need.begin(), need.end(), v) != need.end() &&
                std::find(next.vars.begin(), next.vars.end(), v) == next.vars.end())
              next.vars.push_back(v);
        if (next.vars.size() > (size_t)kMaxK) return fail(CDL_E_INVALID, "intermediate too wide");
        js.out_k = (uint32_t)next.vars.size();
        for (uint32_t k = 0; k < js.out_k; ++k) {
          js.out[k] = ref_of(next.vars[k]);
          const Src& from = js.out[k].side == 0 ? P : B;
          next.bits.push_back(from.bits[js.out[k].v]);
        }
      }
      const bool filter = js.n_neq > 0 || js.n_eq > 0;
      // features of this join, for the estimator's prediction and its log
      const std::tuple<size_t, size_t, size_t> step_key{(size_t)(&rule - rules.data()), start, t};
      // a prediction pays off where the count pass it saves is not trivial
      // (a dense head needs no buffer sized: its tuples become bits)
      const bool predict = ix != nullptr && !js.star && est_ready() && !force_exact &&
                           !(last && rels[rule.head.rel]->dset.words) &&
                           P.n >= (opt.est_min_rows ? opt.est_min_rows : kPredictMinRows);
      const bool feats = ix != nullptr && !js.star && (predict || opt.estimator >= 2);
      auto features = [&]() {
        const Relation* PR = P.rel >= 0 ? rels[P.rel].get() : nullptr;
        const auto po = prev_out.find(step_key);
        return JoinFeatureHost{(float)(PR ? PR->full.n : P.n), (float)ix->distinct,
                               (float)cur_round, po == prev_out.end() ? 0.f : (float)po->second,
                               (float)rels[rule.head.rel]->delta.n, filter ? 1.f : 0.f};
      };
      if (est_plan) {  // planning pass: the features of a first join that writes a head
        if (predict && last && t == 1 && est_nb < kEstBatch) {
          float* X = static_cast<float*>(est_bio.p) + (size_t)est_nb * kMlpIn;
          cudaError_t e = join_features(ctx, P.c[js.pk0], js.pk1 == 0xFFu ? nullptr : P.c[js.pk1],
                                        P.n, ix->cols[hkey[0]],
                                        hkey.size() > 1 ? ix->cols[hkey[1]] : nullptr, B.n,
                                        features(), X);
          if (e != cudaSuccess) return cuda_fail(e, "join features");
          est_slot[step_key] = est_nb++;
        }
        return CDL_OK;
      }
      // predicted in the round's batch: no launch, no wait here
      const auto bslot = est_slot.find(step_key);
      const bool batched = predict && last && bslot != est_slot.end() &&
                           deferred.size() < kMaxDeferred;
      if (feats && batched) {
        std::copy(h_batch + (size_t)bslot->second * kMlpIn,
                  h_batch + (size_t)(bslot->second + 1) * kMlpIn, h_est);
        h_est[kMlpIn] = h_batch[(size_t)kEstBatch * kMlpIn + bslot->second];
      } else if (feats) {
        const JoinFeatureHost hf = features();
        float* io = static_cast<float*>(est_io.p);
        cudaError_t e = join_features(ctx, P.c[js.pk0], js.pk1 == 0xFFu ? nullptr : P.c[js.pk1],
                                      P.n, ix->cols[hkey[0]],
                                      hkey.size() > 1 ? ix->cols[hkey[1]] : nullptr, B.n, hf, io);
        if (e == cudaSuccess && predict)
          e = mlp_infer_bf16(ctx, est_wb.p, io, 1, io + kMlpIn);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(h_est, io, sizeof(float) * (kMlpIn + 1), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "join features");
      }
      auto log_sample = [&](uint64_t size) {
        prev_out[step_key] = size;
        if (!feats || opt.estimator < 2) return;
        log_x.insert(log_x.end(), h_est, h_est + kMlpIn);
        log_y.push_back((float)std::log2(1.0 + (double)size));
      };
      if (predict) {
        // single pass into a buffer sized by the prediction; a batched one
        // sizes it from the host's bound on the cursor instead of reading it
        if (!batched) {
          r = fetch(kSlotScratch, kSlotCursor + (uint32_t)rels.size() - kSlotScratch);
          if (r != CDL_OK) return r;
          note_cursors();
        }
        if (last && rels[rule.head.rel]->fresh_overflow) return CDL_OK;  // redone exact
        const double want =
            std::exp2(std::min(40.0, (double)h_est[kMlpIn] + est_margin + est_boost));
        // a large predicted join keeps the count pass: next to its write the
        // count is cheap, while an overflow would cost the whole round
        if (want <= (opt.est_max_rows ? (double)opt.est_max_rows : kDirectMaxTuples)) {
          const uint64_t cap = std::max<uint64_t>(256, (uint64_t)std::ceil(want));
          Relation* H = last ? rels[rule.head.rel].get() : nullptr;
          const uint64_t cur0 = !last ? 0
                                : batched ? H->fresh_ub
                                          : h_ctl[kSlotCursor + rule.head.rel];
          uint64_t* cursor = dslot(last ? kSlotCursor + rule.head.rel : kSlotAux);
          bool room = true;
          ColsOut out{};
          uint64_t out_cap = 0;
          if (last) {
            H->fresh_ub = cur0;
            room = ensure_fresh(*H, cap) == CDL_OK;
            out = H->fresh.out();
            out_cap = H->fresh.cap;
          } else {
            next.k = js.out_k;
            room = alloc_cols(next.owned, next.k, cap);
            out = next.owned.out();
            out_cap = cap;
          }
          if (room && last && deferred.size() < kMaxDeferred) {
            // no wait: the round's end reads the size and the overflow flag
            const uint32_t di = (uint32_t)deferred.size();
            cudaError_t e = cudaMemsetAsync(heavy.n, 0, 8, st);
            if (e == cudaSuccess)
              e = join_direct(ctx, js, out, cursor, out_cap, static_cast<uint64_t*>(join_sizes.p) + di,
                              reinterpret_cast<uint32_t*>(dslot(kSlotRoundOverflow)), heavy);
            if (e != cudaSuccess) return cuda_fail(e, "single-pass join");
            Deferred d;
            d.step = step_key;
            d.head = rule.head.rel;
            std::copy(h_est, h_est + kMlpIn, d.feat);
            deferred.push_back(d);
            ++est_pred;
            ++joins;
            return CDL_OK;
          }
          if (room) {
            cudaError_t e = cudaMemsetAsync(dslot(kSlotDirTotal), 0, 16, st);  // total, overflow
            if (e == cudaSuccess && !last) e = cudaMemsetAsync(cursor, 0, 8, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(heavy.n, 0, 8, st);
            if (e == cudaSuccess)
              e = join_direct(ctx, js, out, cursor, out_cap, dslot(kSlotDirTotal),
                              reinterpret_cast<uint32_t*>(dslot(kSlotOverflow)), heavy);
            if (e != cudaSuccess) return cuda_fail(e, "single-pass join");
            r = fetch(kSlotDirTotal, 2);
            if (r != CDL_OK) return r;
            const uint64_t total = h_ctl[kSlotDirTotal];
            if (h_ctl[kSlotOverflow] == 0) {
              ++est_pred;
              ++joins;
              log_sample(total);
              if (last) return CDL_OK;
              r = fetch(kSlotAux, 1);
              if (r != CDL_OK) return r;
              next.n = next.owned.n = h_ctl[kSlotAux];
              for (uint32_t k = 0; k < next.k; ++k) next.c[k] = next.owned.c[k];
              if (next.n == 0) return CDL_OK;
              left = std::move(next);
              continue;
            }
          }
          // the prediction was too small: undo the claims, then the exact join
          // (a batched one claimed nothing: it always takes the path above
          // when its buffer has room)
          ++est_over;
          if (last && !batched) {
            h_ctl[kSlotScratch] = cur0;
            cudaError_t e = cudaMemcpyAsync(cursor, h_ctl + kSlotScratch, 8, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "cursor rollback");
            H->fresh_ub = cur0;
          } else {
            next.owned.clear();
          }
        }
      }
      // passes 1 and 2: counts, offsets, total
      DBuf off = alloc(std::max<uint64_t>(P.n, 1) * 8);
      DBuf ws = alloc(join_count_workspace(P.n));
      if (!off.p || !ws.p) return fail(CDL_E_NOMEM, "join offsets");
      // the probe cost per row measures the index's load factor for the tuner
      Tuner::Probe tp;
      // (a star join's count measures it where one index serves both sides)
      if (ix && (!js.star || ix2 == ix) && !ix->tkey.empty() && tuner.mode == 2 && P.n >= 4096) {
        auto& ts = tuner.table[ix->tkey];
        if ((size_t)ix->tcand < ts.size() && ts[ix->tcand].n < Tuner::kTrials)
          tp = tuner.start(ix->tkey, ix->tcand, (double)P.n, st);
      }
      cudaError_t e = join_count_scan(ctx, js, static_cast<uint64_t*>(off.p), dslot(kSlotScratch),
                                      ws.p);
      if (e != cudaSuccess) return cuda_fail(e, "join count");
      tuner.stop(tp, st);
      r = fetch(kSlotScratch, kSlotCursor + (uint32_t)rels.size() - kSlotScratch);
      if (r != CDL_OK) return r;
      note_cursors();
      if (last && !force_exact && rels[rule.head.rel]->fresh_overflow) return CDL_OK;
      const uint64_t total = h_ctl[kSlotScratch];
      ++joins;
      log_sample(total);
      if (recording) {  // a step of a capturable plan: hash join, static build side
        GStep g;
        g.rule = (size_t)(&rule - rules.data());
        g.t = t;
        g.js = js;
        g.last = last;
        g.filter = filter;
        g.head = rule.head.rel;
        g.probe_rel = t == 1 ? P.rel : -1;
        g.seen_probe = P.n;
        g.seen_total = total;
        const bool first_ok = t > 1 || (P.rel >= 0 && P.ver == kDelta && rels[P.rel]->idb);
        const bool later_ok = t == 1 || P.rel < 0;
        if (!ix || &P != &left || B.rel < 0 || rels[B.rel]->idb || !first_ok || !later_ok ||
            (C && (C->rel < 0 || rels[C->rel]->idb)))
          grec_bad = true;
        grec.push_back(g);
      }
      if (total == 0) return CDL_OK;
      ws.reset();
      const size_t wws = join_write_workspace(P.n, total);
      DBuf wsp = alloc(wws);
      if (!wsp.p) return fail(CDL_E_NOMEM, "join splits");
      if (last && rels[rule.head.rel]->dset.words) {  // a dense head: bits, not rows
        Relation& H = *rels[rule.head.rel];
        H.dense_ub += total;
        e = join_write(ctx, js, static_cast<const uint64_t*>(off.p), total, ColsOut{}, 0, nullptr,
                       0, wsp.p, wws, nullptr, nullptr, nullptr, &H.dset);
        if (e != cudaSuccess) return cuda_fail(e, "join write");
        return CDL_OK;
      }
      if (last) {
        Relation& H = *rels[rule.head.rel];
        H.fresh_ub = h_ctl[kSlotCursor + rule.head.rel];
        const uint64_t base = H.fresh_ub;
        r = ensure_fresh(H, total);
        if (r != CDL_OK) return r;
        e = join_write(ctx, js, static_cast<const uint64_t*>(off.p), total, H.fresh.out(), base,
                       dslot(kSlotCursor + rule.head.rel), H.fresh.cap, wsp.p, wws);
        if (e != cudaSuccess) return cuda_fail(e, "join write");
        return CDL_OK;
      }
      next.k = js.out_k;
      if (!alloc_cols(next.owned, next.k, total)) return fail(CDL_E_NOMEM, "join intermediate");
      for (uint32_t k = 0; k < next.k; ++k) next.c[k] = next.owned.c[k];
      e = cudaMemsetAsync(dslot(kSlotAux), 0, 8, st);
      if (e == cudaSuccess)
        e = join_write(ctx, js, static_cast<const uint64_t*>(off.p), total, next.owned.out(), 0,
                       dslot(kSlotAux), total, wsp.p, wws);
      if (e != cudaSuccess) return cuda_fail(e, "join write");
      if (filter) {
        r = fetch(kSlotAux, 1);
        if (r != CDL_OK) return r;
        next.n = h_ctl[kSlotAux];
      } else {
        next.n = total;
      }
      next.owned.n = next.n;
      if (next.n == 0) return CDL_OK;
      left = std::move(next);
    }
    return CDL_OK;
  }

  // A body atom that reads its relation's columns as they are (distinct
  // variables only): its source needs no selection kernel.
  static bool plain_atom(const AtomR& a) {
    for (size_t i = 0; i < a.t.size(); ++i) {
      if (a.t[i].is_const) return false;
      for (size_t j = 0; j < i; ++j)
        if (a.t[j].v == a.t[i].v) return false;
    }
    return true;
  }

  cdl_status eval_rule(const RuleR& rule, bool first_round) {
    // the planning pass takes two-atom rules over plain atoms: their first
    // join writes the head, and setting it up launches nothing
    if (est_plan && (rule.body.size() != 2 || !plain_atom(rule.body[0]) ||
                     !plain_atom(rule.body[1])))
      return CDL_OK;
    // a head relation already marked for an exact redo gains nothing more now
    if (!force_exact && rels[rule.head.rel]->fresh_overflow) return CDL_OK;
    const size_t nb = rule.body.size();
    if (first_round) {
      if (nb == 1) return eval_copy(rule, kFull);
      return eval_join(rule, std::vector<int>(nb, kFull), 0);
    }
    for (size_t i = 0; i < nb; ++i) {
      const Relation& R = *rels[rule.body[i].rel];
      if (!R.idb || R.delta.n == 0) continue;
      std::vector<int> vers(nb, kFull);
      vers[i] = kDelta;
      cdl_status r = nb == 1 ? eval_copy(rule, kDelta) : eval_join(rule, vers, i);
      if (r != CDL_OK) return r;
    }
    return CDL_OK;
  }

  // Derived relations whose tuple space has at most 2^dense_bits tuples (not
  // batched) get a bitmap of that space, empty between rounds.
  cdl_status setup_dense() {
    const int dmax = opt.dense_bits == 0 ? kDenseBits : opt.dense_bits;
    for (auto& rp : rels) {
      Relation& R = *rp;
      R.dset = DenseSet{};
      R.dset_buf.reset();
      R.dense_rows.clear();
      if (!R.idb || opt.n_instances || dmax <= 0 || R.arity == 0) continue;
      uint32_t bits[kMaxK], T = 0;
      for (uint32_t k = 0; k < R.arity; ++k) T += bits[k] = bits_of(R.bound[k]);
      if (T > (uint32_t)std::min(dmax, kDenseBitsMax)) continue;
      const uint64_t nw = T >= 5 ? (1ull << (T - 5)) : 1;
      R.dset_buf = alloc(4 * nw);
      if (!R.dset_buf.p) return fail(CDL_E_NOMEM, "dense set");
      cudaError_t e = cudaMemsetAsync(R.dset_buf.p, 0, 4 * nw, st);
      if (e != cudaSuccess) return cuda_fail(e, "dense set");
      R.dset.words = static_cast<uint32_t*>(R.dset_buf.p);
      R.dset.nbits = 1ull << T;
      R.dset.k = R.arity;
      uint32_t sh = 0;
      for (int k = (int)R.arity - 1; k >= 0; --k) {
        R.dset.shift[k] = sh;
        R.dset.mask[k] = (uint32_t)((1ull << bits[k]) - 1);
        sh += bits[k];
      }
    }
    return CDL_OK;
  }

  // Upper bounds of every column's values: loaded maxima and rule constants,
  // propagated through the rules to a fixpoint.
  void propagate_bounds() {
    bool changed = true;
    while (changed) {
      changed = false;
      for (const RuleR& rule : rules) {
        std::map<uint32_t, uint32_t> vb;
        for (const AtomR& a : rule.body)
          for (uint32_t k = 0; k < a.t.size(); ++k)
            if (!a.t[k].is_const) {
              const uint32_t b = rels[a.rel]->bound[k];
              auto it = vb.find(a.t[k].v);
              if (it == vb.end())
                vb[a.t[k].v] = b;
              else
                it->second = std::min(it->second, b);
            }
        Relation& H = *rels[rule.head.rel];
        for (uint32_t k = 0; k < rule.head.t.size(); ++k) {
          const Term& tm = rule.head.t[k];
          const uint32_t b = tm.is_const ? tm.v : vb[tm.v];
          if (b > H.bound[k]) {
            H.bound[k] = b;
            changed = true;
          }
        }
      }
    }
  }

  // ------------------------------------------------------- batched runs
  // Segment list for gather_segments; adjacent rows of one table coalesce.
  struct Segs {
    std::vector<uint64_t> off{0}, src;
    void add(uint64_t from, uint64_t rows) {
      if (!rows) return;
      if (!src.empty()) {
        const uint64_t last = src.back(), len = off.back() - off[off.size() - 2];
        if ((last >> 63) == (from >> 63) && last + len == from) {
          off.back() += rows;
          return;
        }
      }
      src.push_back(from);
      off.push_back(off.back() + rows);
    }
    uint64_t total() const { return off.back(); }
  };

  cdl_status gather(const Segs& sg, uint32_t k, ColsIn a, ColsIn b, ColsOut out) {
    if (sg.src.empty()) return CDL_OK;
    DBuf d = alloc(8 * (sg.off.size() + sg.src.size()));
    if (!d.p) return fail(CDL_E_NOMEM, "segment table");
    uint64_t* doff = static_cast<uint64_t*>(d.p);
    uint64_t* dsrc = doff + sg.off.size();
    cudaError_t e = cudaMemcpyAsync(doff, sg.off.data(), 8 * sg.off.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dsrc, sg.src.data(), 8 * sg.src.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = gather_segments(ctx, k, a, b, doff, dsrc, (uint32_t)sg.src.size(), sg.total(), out);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host tables die here
    return e == cudaSuccess ? CDL_OK : cuda_fail(e, "gather segments");
  }

  // Rows [bounds[i], bounds[i+1]) of each listed relation's full hold instance i.
  cdl_status full_bounds(const std::vector<Relation*>& rs, std::vector<uint64_t>& hb) {
    const uint32_t ni = opt.n_instances;
    hb.assign((size_t)(ni + 1) * rs.size(), 0);
    if (rs.empty()) return CDL_OK;
    DBuf d = alloc(8 * hb.size());
    if (!d.p) return fail(CDL_E_NOMEM, "instance bounds");
    cudaError_t e = cudaSuccess;
    for (size_t j = 0; j < rs.size() && e == cudaSuccess; ++j)
      e = instance_bounds(ctx, rs[j]->full.c[0], rs[j]->full.n, ni,
                          static_cast<uint64_t*>(d.p) + j * (ni + 1));
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), d.p, 8 * hb.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? CDL_OK : cuda_fail(e, "instance bounds");
  }

  // An instance without a new tuple in any derived relation this round has
  // reached its own fixpoint (instances share no tuples, and every rule
  // joins its atoms on the instance column), so its rows can leave full:
  // later rounds then merge only the instances still running.  The pass
  // runs once the rows waiting to leave are at least 1/8 of full.
  cdl_status retire(uint64_t round) {
    const uint32_t ni = opt.n_instances;
    cudaError_t e = cudaMemcpyAsync(h_inst.data(), inst_last.p, 8 * ni, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "instance marks");
    bool any = false;
    for (uint32_t i = 0; i < ni; ++i)
      if (inst_live[i] && !inst_conv[i] && h_inst[i] != round) inst_conv[i] = any = true;
    if (!any) return CDL_OK;
    std::vector<Relation*> rs;
    for (auto& r : rels)
      if (r->idb && r->full.n) rs.push_back(r.get());
    std::vector<uint64_t> hb;
    cdl_status st_ = full_bounds(rs, hb);
    if (st_ != CDL_OK) return st_;
    uint64_t waiting = 0, rows = 0;
    for (size_t j = 0; j < rs.size(); ++j) {
      rows += rs[j]->full.n;
      for (uint32_t i = 0; i < ni; ++i)
        if (inst_live[i] && inst_conv[i]) waiting += hb[j * (ni + 1) + i + 1] - hb[j * (ni + 1) + i];
    }
    if (waiting * 8 < rows) return CDL_OK;
    for (size_t j = 0; j < rs.size(); ++j) {
      Relation& R = *rs[j];
      const uint64_t* b = hb.data() + j * (ni + 1);
      Segs keep, out;
      for (uint32_t i = 0; i < ni; ++i) {
        const uint64_t cnt = b[i + 1] - b[i];
        if (!inst_live[i] || !cnt) continue;
        if (inst_conv[i]) {
          R.ret_off[i] = R.retired.n + out.total();
          R.ret_cnt[i] = cnt;
          out.add(b[i], cnt);
        } else {
          keep.add(b[i], cnt);
        }
      }
      if (!out.total()) continue;
      const uint64_t need = R.retired.n + out.total();
      if (need > R.retired.cap) {
        DCols grown;
        if (!alloc_cols(grown, R.arity, std::max<uint64_t>(need, R.retired.cap + R.retired.cap / 2)))
          return fail(CDL_E_NOMEM, "retired rows");
        for (uint32_t k = 0; k < R.arity && R.retired.n; ++k) {
          e = cudaMemcpyAsync(grown.c[k], R.retired.c[k], 4 * R.retired.n, cudaMemcpyDeviceToDevice, st);
          if (e != cudaSuccess) return cuda_fail(e, "retired rows");
        }
        grown.n = R.retired.n;
        R.retired = std::move(grown);
      }
      ColsOut tail = R.retired.out();
      for (uint32_t k = 0; k < R.arity; ++k) tail.c[k] += R.retired.n;
      st_ = gather(out, R.arity, R.full.in(), R.full.in(), tail);
      if (st_ != CDL_OK) return st_;
      R.retired.n = need;
      DCols kept;
      if (!alloc_cols(kept, R.arity, keep.total())) return fail(CDL_E_NOMEM, "kept rows");
      st_ = gather(keep, R.arity, R.full.in(), R.full.in(), kept.out());
      if (st_ != CDL_OK) return st_;
      kept.n = keep.total();
      R.full = std::move(kept);
      R.version[kFull]++;
    }
    for (uint32_t i = 0; i < ni; ++i)
      if (inst_conv[i]) inst_live[i] = 0;
    return CDL_OK;
  }

  // Puts retired rows back: full becomes every instance's rows in instance
  // order, the lexicographic order of the whole relation.
  cdl_status assemble() {
    const uint32_t ni = opt.n_instances;
    std::vector<Relation*> rs;
    for (auto& r : rels)
      if (r->idb && r->retired.n) rs.push_back(r.get());
    std::vector<uint64_t> hb;
    cdl_status st_ = full_bounds(rs, hb);
    if (st_ != CDL_OK) return st_;
    for (size_t j = 0; j < rs.size(); ++j) {
      Relation& R = *rs[j];
      const uint64_t* b = hb.data() + j * (ni + 1);
      Segs all;
      for (uint32_t i = 0; i < ni; ++i) {
        if (R.ret_cnt[i])
          all.add(R.ret_off[i] | (1ull << 63), R.ret_cnt[i]);
        else
          all.add(b[i], b[i + 1] - b[i]);
      }
      DCols whole;
      if (!alloc_cols(whole, R.arity, all.total())) return fail(CDL_E_NOMEM, "assembled relation");
      st_ = gather(all, R.arity, R.full.in(), R.retired.in(), whole.out());
      if (st_ != CDL_OK) return st_;
      whole.n = all.total();
      R.full = std::move(whole);
      R.retired.clear();
      R.version[kFull]++;
    }
    return CDL_OK;
  }

  // Batched runs: column 0 of every atom is one variable of the rule (the
  // instance), and loaded instance ids are below n_instances.
  cdl_status check_batched() {
    for (const RuleR& rule : rules) {
      const Term& h = rule.head.t.empty() ? Term{true, 0} : rule.head.t[0];
      bool ok = !h.is_const;
      for (const AtomR& a : rule.body) ok &= !a.t.empty() && !a.t[0].is_const && a.t[0].v == h.v;
      if (!ok) return fail(CDL_E_INVALID, "batched rules must share the instance variable in column 0");
    }
    for (auto& r : rels)
      if (r->arity == 0 || (r->full.n && r->bound[0] >= opt.n_instances))
        return fail(CDL_E_VALUE, "relation " + r->name + " holds an instance id >= n_instances");
    return CDL_OK;
  }

  // Where a head relation's buffer may already be overrun by a predicted join
  // (whose check waits for the round's end), an appending selection reports
  // running out of room in the round's overflow word, not as an error: the
  // relation is then redone exact.
  uint32_t* soft_overflow() {
    return est_ready() && !force_exact ? reinterpret_cast<uint32_t*>(dslot(kSlotRoundOverflow))
                                       : nullptr;
  }

  // A claim past a head relation's buffer (the cursor counts every claim)
  // marks that relation's round for a redo; read after every cursor fetch.
  void note_cursors() {
    for (uint32_t i = 0; i < rels.size(); ++i) {
      Relation& R = *rels[i];
      if (R.idb && h_ctl[kSlotCursor + i] > R.fresh.cap) R.fresh_overflow = true;
    }
  }

  // A round's new tuples of several relations of one arity, each at most
  // kGroupRows, are sorted as one (as grouped loads are): a leading column
  // numbers the relation, so one sort replaces one per relation, and each
  // relation's rows come out as a contiguous, sorted segment whose bounds
  // are the known row counts.  rows[i] then views relation i's segment in
  // one of bufs.
  cdl_status sort_groups(std::vector<DCols>& bufs, std::vector<DCols>& rows,
                         std::vector<uint8_t>& grouped) {
    for (uint32_t k = 1; k < (uint32_t)kMaxK; ++k) {
      std::vector<uint32_t> grp;
      for (uint32_t i = 0; i < rels.size(); ++i) {
        const Relation& R = *rels[i];
        const uint64_t n = h_ctl[kSlotCursor + i];
        if (R.idb && !R.dset.words && R.arity == k && n > 0 && n <= kGroupRows &&
            n <= R.fresh.cap && R.full.n + n <= 0xFFFFFFFFull)
          grp.push_back(i);
      }
      if (grp.size() < kGroupMin) continue;
      const uint32_t ng = (uint32_t)grp.size();
      std::vector<uint64_t> off{0};
      std::vector<ColsIn> src;
      uint32_t bits[kMaxK] = {bits_of(ng - 1), 0, 0, 0};
      for (uint32_t i : grp) {
        const Relation& R = *rels[i];
        off.push_back(off.back() + h_ctl[kSlotCursor + i]);
        src.push_back(R.fresh.in());
        for (uint32_t c = 0; c < k; ++c) bits[c + 1] = std::max(bits[c + 1], bits_of(R.bound[c]));
      }
      DCols comb;
      DBuf dsrc = alloc(sizeof(ColsIn) * ng), doff = alloc(8 * off.size());
      if (!alloc_cols(comb, k + 1, off.back()) || !dsrc.p || !doff.p)
        return fail(CDL_E_NOMEM, "grouped sort");
      comb.n = off.back();
      cudaError_t e = cudaMemcpyAsync(dsrc.p, src.data(), sizeof(ColsIn) * ng,
                                      cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(doff.p, off.data(), 8 * off.size(), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = concat_segments(ctx, comb.out(), static_cast<const ColsIn*>(dsrc.p), k,
                            static_cast<const uint64_t*>(doff.p), ng, comb.n);
      if (e != cudaSuccess) return cuda_fail(e, "grouped sort");
      cdl_status r = sort_cols(comb, bits);
      if (r != CDL_OK) return r;
      for (uint32_t g = 0; g < ng; ++g) {
        DCols& v = rows[grp[g]];
        v.k = k;
        v.n = v.cap = off[g + 1] - off[g];
        for (uint32_t c = 0; c < k; ++c) v.c[c] = comb.c[c + 1] + off[g];
        grouped[grp[g]] = 1;
      }
      bufs.push_back(std::move(comb));
    }
    return CDL_OK;
  }

  // Dense relations at a round's end: the rows written to fresh (copies,
  // single-pass joins) set their bits too, then the bits come out as the
  // round's sorted unique new rows, whose numbers are read back at once.
  cdl_status extract_dense() {
    const uint32_t nr = (uint32_t)rels.size();
    bool any = false;
    for (uint32_t i = 0; i < nr; ++i) {
      Relation& R = *rels[i];
      R.dense_rows.clear();
      if (!R.idb || !R.dset.words) continue;
      const uint64_t nf = std::min<uint64_t>(h_ctl[kSlotCursor + i], R.fresh.cap);
      if (nf == 0 && R.dense_ub == 0) continue;
      const uint64_t cap = std::min<uint64_t>(R.dset.nbits, nf + R.dense_ub);
      DBuf ws = alloc(dense_extract_workspace(R.dset.nbits));
      if (!alloc_cols(R.dense_rows, R.arity, cap) || !ws.p) return fail(CDL_E_NOMEM, "dense rows");
      cudaError_t e = dense_insert(ctx, R.dset, R.fresh.in(), nf);
      if (e == cudaSuccess)
        e = dense_extract(ctx, R.dset, R.dense_rows.out(), cap, dslot(kSlotDelta + i), ws.p);
      if (e != cudaSuccess) return cuda_fail(e, "dense rows");
      any = true;
    }
    if (!any) return CDL_OK;
    cdl_status r = fetch(kSlotDelta, nr);
    if (r != CDL_OK) return r;
    for (uint32_t i = 0; i < nr; ++i) {
      Relation& R = *rels[i];
      if (!R.dense_rows.buf.p) continue;
      R.dense_rows.n = h_ctl[kSlotDelta + i];
      prof.add_bytes(kDense, 4.0 * R.arity * R.dense_rows.n);
    }
    return CDL_OK;
  }

  // Every rule once; then the cursors (and the deferred joins' sizes) are
  // read back.  A relation whose predicted joins claimed past its buffer has
  // only appended to that buffer: its rules run again, exact, from an empty
  // buffer; the other relations keep their tuples.
  cdl_status eval_round(uint64_t round) {
    const uint32_t nr = (uint32_t)rels.size();
    deferred.clear();
    force_exact = false;
    est_slot.clear();
    est_nb = 0;
    cudaError_t e = cudaMemsetAsync(dslot(kSlotCursor), 0, 8 * nr, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dslot(kSlotRoundOverflow), 0, 8, st);
    if (e == cudaSuccess && est_ready()) e = cudaMemsetAsync(join_sizes.p, 0, 8 * kMaxDeferred, st);
    if (e != cudaSuccess) return cuda_fail(e, "round reset");
    for (auto& r : rels) {
      r->fresh_ub = 0;
      r->fresh_overflow = false;
      r->dense_ub = 0;
    }
    if (est_ready() && est_bio.p) {  // the round's predictions, with one wait
      est_plan = true;
      cdl_status s = CDL_OK;
      for (const RuleR& rule : rules)
        if ((s = eval_rule(rule, round == 1)) != CDL_OK) break;
      est_plan = false;
      if (s != CDL_OK) return s;
      if (est_nb) {
        float* X = static_cast<float*>(est_bio.p);
        e = mlp_infer_bf16(ctx, est_wb.p, X, est_nb, X + (size_t)kEstBatch * kMlpIn);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(h_batch, X, sizeof(float) * kMlpIn * est_nb, cudaMemcpyDeviceToHost,
                              st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(h_batch + (size_t)kEstBatch * kMlpIn, X + (size_t)kEstBatch * kMlpIn,
                              sizeof(float) * est_nb, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "round predictions");
        s = fetch(0, 0);
        if (s != CDL_OK) return s;
      }
    }
    for (const RuleR& rule : rules) {
      cdl_status s = eval_rule(rule, round == 1);
      if (s != CDL_OK) return s;
    }
    cdl_status s = fetch(kSlotRoundOverflow, kSlotCursor + nr - kSlotRoundOverflow);
    if (s != CDL_OK) return s;
    note_cursors();
    std::vector<bool> redo(nr, false);
    bool any = false;
    for (uint32_t i = 0; i < nr; ++i)
      if (rels[i]->fresh_overflow) redo[i] = any = true;
    if (!deferred.empty()) {  // exact sizes of the predicted joins
      std::vector<uint64_t> sz(deferred.size());
      e = cudaMemcpyAsync(sz.data(), join_sizes.p, 8 * sz.size(), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "join sizes");
      for (size_t i = 0; i < deferred.size(); ++i) {
        if (deferred[i].head < nr && redo[deferred[i].head]) continue;  // measured again
        prev_out[deferred[i].step] = sz[i];
        if (opt.estimator >= 2) {
          log_x.insert(log_x.end(), deferred[i].feat, deferred[i].feat + kMlpIn);
          log_y.push_back((float)std::log2(1.0 + (double)sz[i]));
        }
      }
    }
    if (!any) return CDL_OK;
    force_exact = true;
    // each overrun widens this run's later predictions by half a step (x 1.41)
    est_boost = std::min(4.0, est_boost + 0.5);
    for (uint32_t i = 0; i < nr; ++i)
      if (redo[i]) {
        ++est_over;
        rels[i]->fresh_ub = 0;
        rels[i]->fresh_overflow = false;
        e = cudaMemsetAsync(dslot(kSlotCursor + i), 0, 8, st);
        if (e != cudaSuccess) return cuda_fail(e, "cursor reset");
      }
    for (const RuleR& rule : rules) {
      if (!redo[rule.head.rel]) continue;
      s = eval_rule(rule, round == 1);
      if (s != CDL_OK) return s;
    }
    force_exact = false;
    s = fetch(kSlotRoundOverflow, kSlotCursor + nr - kSlotRoundOverflow);
    if (s != CDL_OK) return s;
    for (uint32_t i = 0; i < nr; ++i)
      if (redo[i] && h_ctl[kSlotCursor + i] > rels[i]->fresh.cap)
        return fail(CDL_E_CAPACITY, "an exact join overflowed its buffer");
    return CDL_OK;
  }

  // ------------------------------------------------- rounds as a CUDA graph
  // The plan recorded in the first semi-naive round can be captured when
  // every rule with a derived relation in its body has exactly one such
  // atom, every other atom is an input relation joined through its hash
  // index, and every derived relation is the head of a recorded chain.
  bool graph_plan() {
    for (auto& r : rels)
      if (r->dsm.on || r->host_full) return false;  // the captured round keeps Full on the device
    if (grec_bad || grec.empty() || opt.estimator) return false;
    std::vector<bool> active(rels.size(), false);
    for (size_t ri = 0; ri < rules.size(); ++ri) {
      const RuleR& rule = rules[ri];
      size_t idb_atoms = 0, var_atoms = 0;
      for (const AtomR& a : rule.body) {
        idb_atoms += rels[a.rel]->idb;
        bool vars = false;
        for (const Term& t : a.t) vars |= !t.is_const;
        var_atoms += vars;
      }
      if (idb_atoms == 0) continue;  // fires in round 1 only
      if (idb_atoms > 1 || rule.body.size() < 2) return false;
      std::vector<const GStep*> chain;
      for (const GStep& g : grec)
        if (g.rule == ri) chain.push_back(&g);
      size_t covered = 1;  // atoms the recorded steps join (a star step joins two)
      for (const GStep* g : chain) covered += 1 + g->js.star;
      if (covered != var_atoms) return false;
      for (size_t i = 0; i < chain.size(); ++i)
        if (chain[i]->t != i + 1 || chain[i]->last != (i + 1 == chain.size())) return false;
      active[rule.head.rel] = true;
    }
    for (size_t i = 0; i < rels.size(); ++i)
      if (rels[i]->idb && !active[i]) return false;
    return true;
  }

  void graph_release() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (ggraph) cudaGraphDestroy(ggraph);
    gexec = nullptr;
    ggraph = nullptr;
    grel.clear();
    gstep.clear();
    gdev.reset();
    gret.reset();
  }

  // Device state layout inside gdev.
  size_t g_off_next() const { return sizeof(GraphRel) * grel.size(); }
  size_t g_off_ctl() const { return 2 * g_off_next(); }
  size_t g_off_cursor() const { return g_off_ctl() + 64; }
  size_t g_off_step() const { return g_off_cursor() + 8 * grel.size(); }
  size_t g_off_round() const { return g_off_step() + 24 * gstep.size(); }
  size_t g_bytes() const { return g_off_round() + 8 * kGraphRounds; }
  char* gbase() const { return static_cast<char*>(gdev.p); }
  GraphRel* g_cur() const { return reinterpret_cast<GraphRel*>(gbase()); }
  GraphRel* g_next() const { return reinterpret_cast<GraphRel*>(gbase() + g_off_next()); }
  GraphCtl* g_ctl() const { return reinterpret_cast<GraphCtl*>(gbase() + g_off_ctl()); }
  uint64_t* g_cursor(size_t r) const { return reinterpret_cast<uint64_t*>(gbase() + g_off_cursor()) + r; }
  uint64_t* g_step(size_t s, int w) const {  // 0 total, 1 base, 2 intermediate rows
    return reinterpret_cast<uint64_t*>(gbase() + g_off_step()) + 3 * s + w;
  }
  uint64_t* g_round() const { return reinterpret_cast<uint64_t*>(gbase() + g_off_round()); }

  // Buffers at the capacities in gcap_*, the relations' current versions
  // copied in, and the round captured into the body of a device-side loop.
  cdl_status graph_build(uint64_t rounds_done, uint64_t iterations) {
    graph_release();
    std::vector<int> slot(rels.size(), -1);
    for (size_t i = 0; i < rels.size(); ++i)
      if (rels[i]->idb) {
        slot[i] = (int)grel.size();
        grel.emplace_back();
        grel.back().rel = (uint32_t)i;
      }
    gstep.resize(grec.size());
    gdev = alloc(g_bytes());
    if (!gdev.p) return fail(CDL_E_NOMEM, "graph state");
    std::vector<GraphRel> cur(grel.size()), next(grel.size());
    for (size_t j = 0; j < grel.size(); ++j) {
      GRelRes& G = grel[j];
      Relation& R = *rels[G.rel];
      G.Ucap = gcap_u[G.rel];
      G.Fcap = gcap_f[G.rel];
      uint32_t bits[kMaxK];
      for (uint32_t k = 0; k < R.arity; ++k) bits[k] = bits_of(R.bound[k]);
      // small capacities: 10-bit digits where they save a pass (fewer graph nodes)
      uint32_t total_bits = 0;
      for (uint32_t k = 0; k < R.arity; ++k) total_bits += bits[k];
      const bool wide = G.Ucap <= (1u << 18) && (total_bits + 9) / 10 < (total_bits + 7) / 8;
      G.plan = make_radix_plan(R.arity, bits, wide ? 10 : digits_for(total_bits), 512);
      G.sorted_in_alt = G.plan.npass % 2 == 1;
      bool ok = true;
      for (int side = 0; side < 2; ++side) {
        ok &= alloc_cols(G.F[side], R.arity, G.Fcap);
        ok &= alloc_cols(G.D[side], R.arity, G.Ucap);
      }
      ok &= alloc_cols(G.fresh, R.arity, G.Ucap) && alloc_cols(G.alt, R.arity, G.Ucap);
      G.sort_ws = alloc(radix_workspace(G.Ucap, G.plan.bits, G.plan.threads));
      G.merge_ws = alloc(diff_merge_workspace(G.Fcap, G.Ucap));
      if (!ok || !G.sort_ws.p || !G.merge_ws.p) return fail(CDL_E_NOMEM, "graph buffers");
      if (R.full.n > G.Fcap || R.delta.n > G.Ucap) return fail(CDL_E_CAPACITY, "graph capacities");
      for (uint32_t k = 0; k < R.arity; ++k) {
        cudaError_t e = cudaSuccess;
        if (R.full.n)
          e = cudaMemcpyAsync(G.F[0].c[k], R.full.c[k], 4 * R.full.n, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && R.delta.n)
          e = cudaMemcpyAsync(G.D[0].c[k], R.delta.c[k], 4 * R.delta.n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "graph state copy");
      }
      cur[j] = GraphRel{G.F[0].in(), G.D[0].in(), R.full.n, R.delta.n};
      next[j] = GraphRel{G.F[1].in(), G.D[1].in(), 0, 0};
    }
    for (size_t s = 0; s < grec.size(); ++s) {
      const GStep& g = grec[s];
      GStepRes& S = gstep[s];
      S.pcap = g.t == 1 ? gcap_u[g.probe_rel] : gstep[s - 1].ocap;
      S.ocap = g.last ? gcap_u[g.head] : gcap_i[s];
      S.off = alloc(8 * S.pcap);
      S.cws = alloc(join_count_workspace(S.pcap));
      S.wbytes = join_write_workspace(S.pcap, S.ocap);
      S.wws = alloc(S.wbytes);
      if (!S.off.p || !S.cws.p || !S.wws.p) return fail(CDL_E_NOMEM, "graph join buffers");
      if (!g.last && !alloc_cols(S.inter, g.js.out_k, S.ocap)) return fail(CDL_E_NOMEM, "graph join buffers");
    }
    if (graph_retires()) {
      cdl_status rr = graph_retire_setup();
      if (rr != CDL_OK) return rr;
    }
    GraphCtl ctl{};
    ctl.round = rounds_done;
    ctl.iterations = iterations;
    ctl.max_iters = opt.max_iters;
    cudaError_t e = cudaMemsetAsync(gdev.p, 0, g_bytes(), st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g_cur(), cur.data(), sizeof(GraphRel) * cur.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g_next(), next.data(), sizeof(GraphRel) * next.size(),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_ctl(), &ctl, sizeof ctl, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "graph state");

    // capture: one round inside a while node whose condition round_end sets
    e = cudaGraphCreate(&ggraph, 0);
    cudaGraphConditionalHandle loop{};
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&loop, ggraph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = loop;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, ggraph, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) return cuda_fail(e, "graph loop node");
    cudaGraph_t body = np.conditional.phGraph_out[0];
    // capture on a stream of its own (the engine's may be the legacy default
    // stream, which cannot capture); the graph is launched on the engine's
    cudaStream_t gst = nullptr;
    e = cudaStreamCreateWithFlags(&gst, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "graph stream");
    Profiler* saved = ctx.prof;
    const cudaStream_t main_st = st;
    Profiler counter;  // counts the captured launches, records no events
    ctx.prof = &counter;
    ctx.st = st = gst;
    e = cudaStreamBeginCaptureToGraph(gst, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) e = graph_round(slot, loop);
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(gst, &captured);
    ctx.prof = saved;
    ctx.st = st = main_st;
    cudaStreamDestroy(gst);
    glaunches_per_round = counter.total_launches;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, ggraph, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "graph capture");
    }
    return CDL_OK;
  }

  // The launches of one round, each reading its sizes (and the current
  // full / delta columns) from the device state.
  cudaError_t graph_round(const std::vector<int>& slot, cudaGraphConditionalHandle loop) {
    uint32_t* ovf = &g_ctl()->overflow;
    cudaError_t e = cudaSuccess;  // the cursors start at 0 (zeroed state, then round_end)
    for (size_t s = 0; s < grec.size() && e == cudaSuccess; ++s) {
      const GStep& g = grec[s];
      GStepRes& S = gstep[s];
      JoinSpec js = g.js;
      js.n_probe = S.pcap;
      if (g.t == 1) {
        GraphRel* c = g_cur() + slot[g.probe_rel];
        js.dprobe = &c->D;
        js.dn = &c->nD;
      } else {
        js.probe = gstep[s - 1].inter.in();
        js.dprobe = nullptr;
        js.dn = g_step(s - 1, 2);
      }
      GRelRes* H = g.last ? &grel[slot[g.head]] : nullptr;
      uint64_t* cursor = g.last ? g_cursor(slot[g.head]) : g_step(s, 2);
      const ColsOut out = g.last ? H->fresh.out() : S.inter.out();
      e = join_count_scan(ctx, js, static_cast<uint64_t*>(S.off.p), g_step(s, 0), S.cws.p);
      if (e == cudaSuccess)
        e = join_write(ctx, js, static_cast<const uint64_t*>(S.off.p), S.ocap, out, 0, cursor,
                       S.ocap, S.wws.p, S.wbytes, g_step(s, 0), g.filter ? nullptr : g_step(s, 1),
                       ovf);
    }
    for (size_t j = 0; j < grel.size() && e == cudaSuccess; ++j) {
      GRelRes& G = grel[j];
      const Relation& R = *rels[G.rel];
      bool in_b = false;
      e = radix_sort(ctx, G.plan, G.fresh.out(), G.alt.out(), G.Ucap, G.sort_ws.p, &in_b,
                     g_cursor(j));
      const DCols& U = G.sorted_in_alt ? G.alt : G.fresh;
      DevMerge dm;
      dm.full = &g_cur()[j].F;
      dm.n_full = &g_cur()[j].nF;
      dm.n_fresh = g_cursor(j);
      dm.delta = reinterpret_cast<const ColsOut*>(&g_next()[j].D);
      dm.merged = reinterpret_cast<const ColsOut*>(&g_next()[j].F);
      dm.cap_merged = G.Fcap;
      dm.overflow = ovf;
      if (e == cudaSuccess)
        e = diff_merge(ctx, R.arity, ColsIn{}, G.Fcap, U.in(), G.Ucap, ColsOut{}, ColsOut{},
                       &g_next()[j].nD, G.merge_ws.p, &dm);
      if (e == cudaSuccess && opt.n_instances)
        e = mark_instances(ctx, nullptr, G.Ucap, opt.n_instances,
                           static_cast<uint64_t*>(inst_last.p), 1, &g_next()[j].D,
                           &g_next()[j].nD, &g_ctl()->round);
    }
    if (e == cudaSuccess)
      e = round_end(ctx, g_cur(), g_next(), (uint32_t)grel.size(), g_ctl(), g_round(), kGraphRounds,
                    loop, g_cursor(0), (uint32_t)grel.size(), g_step(0, 0), (uint32_t)gstep.size());
    if (e == cudaSuccess && graph_retires()) {
      std::vector<uint32_t> ar(grel.size());
      for (size_t j = 0; j < grel.size(); ++j) ar[j] = rels[grel[j].rel]->arity;
      e = retire_round(ctx, g_cur(), g_next(), g_ctl(), g_rctl(), g_rrel(), ar.data(),
                       (uint32_t)grel.size(), opt.n_instances,
                       static_cast<const uint64_t*>(inst_last.p));
    }
    return e;
  }

  // The retirement state of a batched graph: the host's flags, retired rows
  // and per-instance places copied to the device (the graph continues them).
  cdl_status graph_retire_setup() {
    const uint32_t ni = opt.n_instances;
    const size_t nrel = grel.size();
    const size_t per_rel = 8 * (size_t)(7 * ni + 3);  // bounds, kseg, rseg (ni + 1); ret, src (ni)
    const size_t bytes = 256 + ((sizeof(RetireRel) * nrel + 255) & ~size_t(255)) + 8 * (size_t)ni +
                         per_rel * nrel + 256;
    gret = alloc(bytes);
    if (!gret.p) return fail(CDL_E_NOMEM, "graph retirement state");
    char* base = static_cast<char*>(gret.p);
    char* p = base + 256 + ((sizeof(RetireRel) * nrel + 255) & ~size_t(255));
    RetireCtl rc{};
    rc.live = reinterpret_cast<uint32_t*>(p);
    rc.conv = rc.live + ni;
    p += 8 * (size_t)ni;
    std::vector<uint32_t> flags(2 * (size_t)ni);
    for (uint32_t i = 0; i < ni; ++i) {
      flags[i] = inst_live[i];
      flags[ni + i] = inst_conv[i];
    }
    cudaError_t e = cudaMemcpyAsync(rc.live, flags.data(), 8 * (size_t)ni, cudaMemcpyHostToDevice, st);
    std::vector<RetireRel> rr(nrel);
    for (size_t j = 0; j < nrel && e == cudaSuccess; ++j) {
      GRelRes& G = grel[j];
      Relation& R = *rels[G.rel];
      uint64_t* a = reinterpret_cast<uint64_t*>(p + per_rel * j);
      RetireRel& q = rr[j];
      q.bounds = a;
      q.kseg_off = a + (ni + 1);
      q.rseg_off = a + 2 * (size_t)(ni + 1);
      q.ret_off = a + 3 * (size_t)(ni + 1);
      q.ret_cnt = q.ret_off + ni;
      q.kseg_src = q.ret_cnt + ni;
      q.rseg_src = q.kseg_src + ni;
      q.ret_cap = std::max<uint64_t>(2 * R.retired.n, gret_room * G.Fcap);
      if (!alloc_cols(G.ret, R.arity, q.ret_cap)) return fail(CDL_E_NOMEM, "graph retired rows");
      q.ret = G.ret.out();
      q.ret_n = R.retired.n;
      for (uint32_t k = 0; k < R.arity && R.retired.n && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(G.ret.c[k], R.retired.c[k], 4 * R.retired.n, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(q.ret_off, R.ret_off.data(), 8 * (size_t)ni, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(q.ret_cnt, R.ret_cnt.data(), 8 * (size_t)ni, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(base, &rc, sizeof rc, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + 256, rr.data(), sizeof(RetireRel) * nrel, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host vectors die here
    return e == cudaSuccess ? CDL_OK : cuda_fail(e, "graph retirement state");
  }

  // The graph's retirement state back to the host (after its launch).
  cdl_status graph_retire_collect() {
    const uint32_t ni = opt.n_instances;
    const size_t nrel = grel.size();
    RetireCtl rc{};
    std::vector<RetireRel> rr(nrel);
    cudaError_t e = cudaMemcpyAsync(&rc, gret.p, sizeof rc, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rr.data(), g_rrel(), sizeof(RetireRel) * nrel, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "graph retirement state");
    std::vector<uint32_t> flags(2 * (size_t)ni);
    e = cudaMemcpy(flags.data(), rc.live, 8 * (size_t)ni, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "graph retirement state");
    for (uint32_t i = 0; i < ni; ++i) {
      inst_live[i] = (uint8_t)flags[i];
      inst_conv[i] = (uint8_t)flags[ni + i];
    }
    if (rc.short_room) gret_room *= 2;
    g_retirements += rc.moves;
    for (size_t j = 0; j < nrel; ++j) {
      GRelRes& G = grel[j];
      Relation& R = *rels[G.rel];
      e = cudaMemcpy(R.ret_off.data(), rr[j].ret_off, 8 * (size_t)ni, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy(R.ret_cnt.data(), rr[j].ret_cnt, 8 * (size_t)ni, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "graph retirement state");
      R.retired = std::move(G.ret);
      R.retired.n = rr[j].ret_n;
    }
    return CDL_OK;
  }

  // Runs rounds on the device until the fixpoint, max_iters or a buffer
  // overflow; then hands the current versions back to the relations.
  cdl_status graph_run(uint64_t& round, std::vector<uint64_t>& per_round, uint64_t& iterations,
                       bool& finished) {
    finished = false;
    for (size_t i = 0; i < rels.size(); ++i) {  // room for the current versions
      const Relation& R = *rels[i];
      if (!R.idb) continue;
      gcap_u[i] = std::max<uint64_t>({gcap_u[i], 8 * R.delta.n, 8 * R.fresh.n});
      gcap_f[i] = std::max<uint64_t>(gcap_f[i], R.full.n + 16 * gcap_u[i]);
    }
    cdl_status r = graph_build(round, iterations);
    if (r == CDL_E_NOMEM || r == CDL_E_CAPACITY) {  // no room for a graph: rounds stay on the host
      graph_release();
      cudaGetLastError();
      graph_ready = false;
      return CDL_OK;
    }
    if (r != CDL_OK) return r;
    ++g_builds;
    cudaError_t e = cudaGraphLaunch(gexec, st);
    GraphCtl ctl{};
    std::vector<GraphRel> cur(grel.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, g_ctl(), sizeof ctl, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cur.data(), g_cur(), sizeof(GraphRel) * cur.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    r = fetch(0, 0);  // the error word of every launch
    if (r != CDL_OK) return r;
    const uint64_t first = round;
    if (ctl.round > first) {
      std::vector<uint64_t> pr(ctl.round - first);
      e = cudaMemcpy(pr.data(), g_round() + first, 8 * pr.size(), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "graph rounds");
      per_round.insert(per_round.end(), pr.begin(), pr.end());
    }
    prof.total_launches += (ctl.round - first + (ctl.done == 2)) * glaunches_per_round;
    g_rounds += ctl.round - first;
    round = ctl.round;
    iterations = ctl.iterations;
    if (graph_retires()) {
      r = graph_retire_collect();
      if (r != CDL_OK) return r;
    }
    for (size_t j = 0; j < grel.size(); ++j) {
      GRelRes& G = grel[j];
      Relation& R = *rels[G.rel];
      const int side = cur[j].F.c[0] == G.F[0].c[0] ? 0 : 1;
      R.full = std::move(G.F[side]);
      R.full.n = cur[j].nF;
      R.delta = std::move(G.D[side]);
      R.delta.n = cur[j].nD;
      R.version[kFull]++;
      R.version[kDelta]++;
    }
    graph_release();
    evict_stale();
    if (ctl.done == 3) return fail(CDL_E_MAXITER, "the fixpoint needs more rounds than max_iters");
    finished = ctl.done == 1;
    if (ctl.done == 2)  // a buffer was too small: the next round runs on the host, then larger
      for (auto& c : gcap_u) c *= 2;
    if (ctl.done == 2) {
      for (auto& c : gcap_i) c *= 2;
      for (size_t i = 0; i < rels.size(); ++i)
        if (rels[i]->idb) gcap_f[i] = std::max(2 * gcap_f[i], rels[i]->full.n + 16 * gcap_u[i]);
    }
    return CDL_OK;
  }

  // Capacities from the recorded round: room for the sizes seen, many times over.
  void graph_caps() {
    gcap_u.assign(rels.size(), 0);
    gcap_f.assign(rels.size(), 0);
    gcap_i.assign(grec.size(), 0);
    std::vector<uint64_t> seen(rels.size(), 0);
    for (const GStep& g : grec)
      if (g.last) seen[g.head] += g.seen_total;
    // option graph >= 2: that many rows at least instead of 2^16 (small
    // values make later rounds outgrow the buffers, as tests want)
    const uint64_t floor = opt.graph >= 2 ? (uint64_t)opt.graph : (1u << 16);
    for (size_t i = 0; i < rels.size(); ++i) {
      if (!rels[i]->idb) continue;
      gcap_u[i] = std::max<uint64_t>({8 * seen[i], 8 * rels[i]->delta.n, floor});
      gcap_f[i] = std::max<uint64_t>(4 * rels[i]->full.n, rels[i]->full.n + 16 * gcap_u[i]);
    }
    for (size_t s = 0; s < grec.size(); ++s)
      gcap_i[s] = std::max<uint64_t>(8 * grec[s].seen_total, floor);
  }

  cdl_status run(cdl_stats* stats) {
    if (ran) return fail(CDL_E_STATE, "cdl_run was already called");
    cdl_status fl = flush_loads();
    if (fl != CDL_OK) return fl;
    ran = true;
    for (auto& r : rels) r->idb = false;
    for (const RuleR& rule : rules) rels[rule.head.rel]->idb = true;
    propagate_bounds();
    cdl_status ds = setup_dense();
    if (ds != CDL_OK) return ds;
    dsm_select();
    prof.reset();
    joins = 0;
    index_merges = 0;
    star_joins = 0;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventRecord(t0, st);
    uint64_t iterations = resume_iters, rounds = resume_rounds;
    std::vector<uint64_t> per_round = resume_per_round;
    const uint64_t first_semi = std::max<uint64_t>(2, resume_rounds + 1);
    cdl_status status = CDL_OK;
    const uint32_t nr = (uint32_t)rels.size();
    est_pred = est_over = 0;
    est_boost = 0.0;
    if (opt.estimator >= 1) {
      constexpr uint64_t kHeavyCap = 1 << 20;  // chunks of 2048 outputs: 2^31 outputs
      join_sizes = alloc(8 * kMaxDeferred);
      heavy_buf = alloc(256 + sizeof(HeavyChunk) * kHeavyCap);
      if (!join_sizes.p || !heavy_buf.p) return fail(CDL_E_NOMEM, "join sizes");
      est_bio = alloc(sizeof(float) * kEstBatch * (kMlpIn + 1));
      if (!est_bio.p || (!h_batch && cudaMallocHost(&h_batch, sizeof(float) * kEstBatch *
                                                                  (kMlpIn + 1)) != cudaSuccess))
        return fail(CDL_E_NOMEM, "round predictions");
      heavy.n = static_cast<uint64_t*>(heavy_buf.p);
      heavy.e = reinterpret_cast<HeavyChunk*>(static_cast<char*>(heavy_buf.p) + 256);
      heavy.cap = kHeavyCap;
    }
    if (opt.n_instances) {
      cdl_status c = check_batched();
      if (c != CDL_OK) return c;
      inst_last = alloc(sizeof(uint64_t) * opt.n_instances);
      if (!inst_last.p) return fail(CDL_E_NOMEM, "instance marks");
      if (cudaMemsetAsync(inst_last.p, 0, sizeof(uint64_t) * opt.n_instances, st) != cudaSuccess)
        return fail(CDL_E_CUDA, "instance marks");
      h_inst.assign(opt.n_instances, 0);
      inst_live.assign(opt.n_instances, 1);
      inst_conv.assign(opt.n_instances, 0);
      for (auto& r : rels) {
        r->ret_off.assign(opt.n_instances, 0);
        r->ret_cnt.assign(opt.n_instances, 0);
      }
    }
    grec.clear();
    grec_bad = graph_ready = false;
    g_rounds = g_builds = g_retirements = 0;
    for (uint64_t round = resume_rounds + 1; status == CDL_OK; ++round) {
      cur_round = round;
      cudaError_t e = cudaSuccess;
      recording = opt.graph && round == first_semi;  // the first semi-naive round is the plan
      status = eval_round(round);
      recording = false;
      if (status == CDL_OK) status = extract_dense();
      if (status != CDL_OK) break;
      // relations of one arity with few new tuples each are sorted as one
      std::vector<DCols> group_bufs, sorted_rows(nr);
      std::vector<uint8_t> grouped(nr, 0);
      if (!opt.n_instances) status = sort_groups(group_bufs, sorted_rows, grouped);
      if (status != CDL_OK) break;
      std::vector<uint8_t> merged(nr, 0);
      for (uint32_t i = 0; i < nr; ++i) {
        Relation& R = *rels[i];
        if (!R.idb) continue;
        R.fresh.n = h_ctl[kSlotCursor + i];
        R.delta.clear();
        R.delta.k = R.arity;
        R.version[kDelta]++;
        e = cudaMemsetAsync(dslot(kSlotDelta + i), 0, 8, st);
        if (e != cudaSuccess) {
          status = cuda_fail(e, "delta reset");
          break;
        }
        if (R.dset.words) {  // the dense form: the round's rows come out sorted and unique
          DCols rows = std::move(R.dense_rows);
          if (rows.n == 0) continue;
          if (R.full.n + rows.n > 0xFFFFFFFFull) {
            status = fail(CDL_E_CAPACITY, "relation " + R.name + " would exceed 2^32 tuples");
            break;
          }
          status = merge_into(R, rows, &R.delta, kSlotDelta + i);
          if (status != CDL_OK) break;
          merged[i] = 1;
          continue;
        }
        if (R.fresh.n == 0) continue;
        if (R.full.n + R.fresh.n > 0xFFFFFFFFull) {
          status = fail(CDL_E_CAPACITY, "relation " + R.name + " would exceed 2^32 tuples");
          break;
        }
        if (grouped[i]) {  // sorted with its group: a segment of the group's rows
          status = merge_into(R, sorted_rows[i], &R.delta, kSlotDelta + i);
          if (status != CDL_OK) break;
          merged[i] = 1;
          continue;
        }
        uint32_t bits[kMaxK];
        for (uint32_t k = 0; k < R.arity; ++k) bits[k] = bits_of(R.bound[k]);
        status = sort_cols(R.fresh, bits);
        if (status != CDL_OK) break;
        status = merge_into(R, R.fresh, &R.delta, kSlotDelta + i);
        if (status != CDL_OK) break;
        merged[i] = 1;
      }
      if (status != CDL_OK) break;
      status = fetch(kSlotDelta, nr);
      if (status != CDL_OK) break;
      uint64_t new_total = 0;
      for (uint32_t i = 0; i < nr; ++i) {
        Relation& R = *rels[i];
        if (!R.idb) continue;
        const uint64_t nd = merged[i] ? h_ctl[kSlotDelta + i] : 0;
        R.delta.n = nd;
        R.full.n += nd;
        if (merged[i] && R.dsm.on) {
          prof.add_bytes(kDedup, 4.0 * R.arity * nd);  // delta written by the compaction
          status = dsm_append(R);
          if (status != CDL_OK) break;
        } else if (merged[i]) {
          prof.add_bytes(kDiffMerge, 8.0 * R.arity * nd);
        }
        new_total += nd;
        if (opt.n_instances && nd) {  // batched: instances that derived in this round
          cudaError_t e = mark_instances(ctx, R.delta.c[0], nd, opt.n_instances,
                                         static_cast<uint64_t*>(inst_last.p), round);
          if (e != cudaSuccess) {
            status = cuda_fail(e, "instance marks");
            break;
          }
        }
      }
      if (status != CDL_OK) break;
      if (opt.n_instances && new_total && opt.retire >= 0) {
        status = retire(round);
        if (status != CDL_OK) break;
      }
      evict_stale();
      tuner.resolve();  // the stream was synchronised by the fetches above
      rounds = round;
      per_round.push_back(new_total);
      if (new_total == 0) break;
      iterations = round;
      if (opt.max_iters && iterations > opt.max_iters) {
        status = fail(CDL_E_MAXITER, "the fixpoint needs more rounds than max_iters");
        break;
      }
      if (opt.graph && round == first_semi) {
        graph_ready = graph_plan();
        if (graph_ready) graph_caps();
      }
      if (graph_ready && round >= first_semi) {  // the next rounds on the device
        bool finished = false;
        status = graph_run(round, per_round, iterations, finished);
        rounds = round;
        if (status != CDL_OK || finished) break;
      }
    }
    graph_release();
    prev_full.clear();
    if (status == CDL_OK || status == CDL_E_MAXITER) {
      const cdl_status fs = dsm_finish();
      if (status == CDL_OK) status = fs;
    }
    if (opt.n_instances && status == CDL_OK) status = assemble();
    last_rounds = rounds;
    last_iters = iterations;
    last_per_round = per_round;
    tuner.resolve();
    if (tuner.mode == 2 && !tuner.save() && status == CDL_OK)
      status = fail(CDL_E_INVALID, "cannot write the tuner file");
    cudaEventRecord(t1, st);
    cudaEventSynchronize(t1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    prof.collect();
    for (auto& r : rels) {
      r->fresh.clear();
      r->fresh_ub = 0;
    }
    if (stats) {
      stats->iterations = iterations;
      stats->rounds = rounds;
      uint64_t derived = 0;
      for (auto& r : rels)
        if (r->idb) derived += r->full.n;
      stats->derived_tuples = derived;
      stats->seconds = ms * 1e-3;
      stats->algo_bytes = prof.total_bytes;
      stats->joins = joins;
      stats->kernel_launches = prof.total_launches;
      stats->est_predictions = est_pred;
      stats->est_overflows = est_over;
      stats->graph_rounds = g_rounds;
      stats->graph_builds = g_builds;
      stats->index_merges = index_merges;
      stats->star_joins = star_joins;
      stats->graph_retirements = g_retirements;
      if (stats->delta_per_round)
        for (uint64_t i = 0; i < per_round.size() && i < stats->delta_cap; ++i)
          stats->delta_per_round[i] = per_round[i];
      if (stats->iters_per_instance && opt.n_instances && inst_last.p && status == CDL_OK) {
        cudaError_t e = cudaMemcpyAsync(stats->iters_per_instance, inst_last.p,
                                        sizeof(uint64_t) * opt.n_instances, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) status = cuda_fail(e, "instance iterations");
      }
    }
    return status;
  }

  // --------------------------------------------------------- checkpoints
  // File: "CDLCKPT1", rounds, iterations, per-round count and sizes, then per
  // relation its name, arity, |full|, |delta| and the columns of full and
  // delta (uint32, host byte order).
  cdl_status checkpoint_save(const char* path) {
    if (!ran) return fail(CDL_E_STATE, "nothing to save before cdl_run");
    if (opt.n_instances) return fail(CDL_E_INVALID, "batched runs are not checkpointed");
    FILE* f = path ? std::fopen(path, "wb") : nullptr;
    if (!f) return fail(CDL_E_INVALID, "cannot write the checkpoint file");
    bool ok = std::fwrite("CDLCKPT1", 1, 8, f) == 8;
    const uint64_t head[3] = {last_rounds, last_iters, (uint64_t)last_per_round.size()};
    ok &= std::fwrite(head, 8, 3, f) == 3;
    ok &= std::fwrite(last_per_round.data(), 8, last_per_round.size(), f) == last_per_round.size();
    const uint32_t nrel = (uint32_t)rels.size();
    ok &= std::fwrite(&nrel, 4, 1, f) == 1;
    std::vector<uint32_t> col;
    for (auto& rp : rels) {
      const Relation& R = *rp;
      const uint32_t nl = (uint32_t)R.name.size();
      const uint64_t sz[2] = {R.full.n, R.delta.n};
      ok &= std::fwrite(&nl, 4, 1, f) == 1 && std::fwrite(R.name.data(), 1, nl, f) == nl;
      ok &= std::fwrite(&R.arity, 4, 1, f) == 1 && std::fwrite(sz, 8, 2, f) == 2;
      for (const DCols* d : {&R.full, &R.delta})
        for (uint32_t k = 0; k < R.arity && ok && d->n; ++k) {
          col.resize(d->n);
          if (cudaMemcpy(col.data(), d->c[k], 4 * d->n, cudaMemcpyDefault) != cudaSuccess) {
            std::fclose(f);
            return fail(CDL_E_CUDA, "checkpoint copy");
          }
          ok &= std::fwrite(col.data(), 4, d->n, f) == d->n;
        }
    }
    ok &= std::fclose(f) == 0;
    return ok ? CDL_OK : fail(CDL_E_INVALID, "checkpoint write failed");
  }

  cdl_status checkpoint_load(const char* path) {
    if (ran) return fail(CDL_E_STATE, "checkpoints load before cdl_run");
    if (opt.n_instances) return fail(CDL_E_INVALID, "batched runs are not checkpointed");
    FILE* f = path ? std::fopen(path, "rb") : nullptr;
    if (!f) return fail(CDL_E_INVALID, "cannot read the checkpoint file");
    auto bad = [&](const char* m) {
      std::fclose(f);
      return fail(CDL_E_INVALID, std::string("checkpoint: ") + m);
    };
    char magic[8];
    uint64_t head[3];
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, "CDLCKPT1", 8) != 0)
      return bad("not a checkpoint");
    if (std::fread(head, 8, 3, f) != 3 || head[2] > (1ull << 32)) return bad("truncated header");
    std::vector<uint64_t> pr(head[2]);
    if (std::fread(pr.data(), 8, pr.size(), f) != pr.size()) return bad("truncated rounds");
    uint32_t nrel = 0;
    if (std::fread(&nrel, 4, 1, f) != 1) return bad("truncated header");
    std::vector<uint32_t> col;
    for (uint32_t i = 0; i < nrel; ++i) {
      uint32_t nl = 0, ar = 0;
      uint64_t sz[2];
      if (std::fread(&nl, 4, 1, f) != 1 || nl > 4096) return bad("truncated relation");
      std::string name(nl, '\0');
      if (std::fread(&name[0], 1, nl, f) != nl || std::fread(&ar, 4, 1, f) != 1 ||
          std::fread(sz, 8, 2, f) != 2)
        return bad("truncated relation");
      auto it = by_name.find(name);
      if (it == by_name.end() || rels[it->second]->arity != ar)
        return bad("relation not declared with that arity");
      Relation& R = *rels[it->second];
      if (sz[0] > 0xFFFFFFFFull || sz[1] > sz[0]) return bad("bad sizes");
      DCols* dst[2] = {&R.full, &R.delta};
      for (int v = 0; v < 2; ++v) {
        DCols& d = *dst[v];
        d.clear();
        if (!alloc_cols(d, ar, std::max<uint64_t>(sz[v], 1))) {
          std::fclose(f);
          return fail(CDL_E_NOMEM, "checkpoint buffers");
        }
        d.n = sz[v];
        for (uint32_t k = 0; k < ar && sz[v]; ++k) {
          col.resize(sz[v]);
          if (std::fread(col.data(), 4, sz[v], f) != sz[v]) return bad("truncated columns");
          if (cudaMemcpy(d.c[k], col.data(), 4 * sz[v], cudaMemcpyHostToDevice) != cudaSuccess) {
            std::fclose(f);
            return fail(CDL_E_CUDA, "checkpoint copy");
          }
        }
      }
      if (R.full.n) {  // column bounds, as a load computes them
        uint32_t* dmax = reinterpret_cast<uint32_t*>(dslot(kSlotScratch + 1));
        cudaError_t e = check_values(ctx, R.full.in(), ar, R.full.n, dmax);
        if (e != cudaSuccess) {
          std::fclose(f);
          return cuda_fail(e, "checkpoint check");
        }
        cdl_status r = fetch(kSlotScratch + 1, 2);
        if (r != CDL_OK) {
          std::fclose(f);
          return r;
        }
        const uint32_t* hmax = reinterpret_cast<const uint32_t*>(h_ctl + kSlotScratch + 1);
        for (uint32_t k = 0; k < ar; ++k) R.bound[k] = std::max(R.bound[k], hmax[k]);
      }
      R.version[kFull]++;
      R.version[kDelta]++;
    }
    std::fclose(f);
    evict_stale();
    resume_rounds = head[0];
    resume_iters = head[1];
    resume_per_round = pr;
    return CDL_OK;
  }

  cdl_status load(uint32_t rel, const uint32_t* const* cols, uint64_t n, int on_device) {
    if (ran) return fail(CDL_E_STATE, "loads must precede cdl_run");
    Relation& R = *rels[rel];
    if (n == 0) return CDL_OK;
    if (n > 0xFFFFFFFFull) return fail(CDL_E_CAPACITY, "load exceeds 2^32 tuples");
    DCols in;
    if (!alloc_cols(in, R.arity, n)) return fail(CDL_E_NOMEM, "load buffer");
    in.n = n;
    for (uint32_t k = 0; k < R.arity; ++k) {
      if (!cols[k]) return fail(CDL_E_INVALID, "null column pointer");
      cudaError_t e = cudaMemcpyAsync(in.c[k], cols[k], n * 4,
                                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                      st);
      if (e != cudaSuccess) return cuda_fail(e, "load copy");
    }
    uint32_t* dmax = reinterpret_cast<uint32_t*>(dslot(kSlotScratch + 1));  // slots 2..3
    cudaError_t e = check_values(ctx, in.in(), R.arity, n, dmax);
    if (e != cudaSuccess) return cuda_fail(e, "load check");
    cdl_status r = fetch(kSlotScratch + 1, 2);
    if (r != CDL_OK) {
      cudaMemsetAsync(dslot(kSlotErr), 0, 8, st);
      return r;
    }
    const uint32_t* hmax = reinterpret_cast<const uint32_t*>(h_ctl + kSlotScratch + 1);
    for (uint32_t k = 0; k < R.arity; ++k) R.bound[k] = std::max(R.bound[k], hmax[k]);
    R.pending.push_back(std::move(in));  // sorted and merged with the others by flush_loads
    return CDL_OK;
  }

  // Several loads with one check: every load's columns are copied and
  // scanned (maxima per column, the reserved value) back to back, then one
  // wait reads all maxima and the error word.  All are added, or none.
  cdl_status load_many(uint32_t count, const cdl_rel* rl, const uint32_t* const* const* cols,
                       const uint64_t* ns, int on_device) {
    if (ran) return fail(CDL_E_STATE, "loads must precede cdl_run");
    for (uint32_t i = 0; i < count; ++i) {
      if (rl[i] >= rels.size()) return fail(CDL_E_INVALID, "no such relation");
      if (ns[i] > 0xFFFFFFFFull) return fail(CDL_E_CAPACITY, "load exceeds 2^32 tuples");
      if (!ns[i]) continue;
      if (!cols[i]) return fail(CDL_E_INVALID, "null column pointer");
      for (uint32_t k = 0; k < rels[rl[i]]->arity; ++k)
        if (!cols[i][k]) return fail(CDL_E_INVALID, "null column pointer");
    }
    DBuf mx = alloc(4 * kMaxK * std::max<uint32_t>(count, 1));
    if (!mx.p) return fail(CDL_E_NOMEM, "load maxima");
    std::vector<DCols> in(count);
    for (uint32_t i = 0; i < count; ++i) {
      if (!ns[i]) continue;
      const uint32_t ar = rels[rl[i]]->arity;
      if (!alloc_cols(in[i], ar, ns[i])) return fail(CDL_E_NOMEM, "load buffer");
      in[i].n = ns[i];
      cudaError_t e = cudaSuccess;
      for (uint32_t k = 0; k < ar && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(in[i].c[k], cols[i][k], ns[i] * 4,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = check_values(ctx, in[i].in(), ar, ns[i], static_cast<uint32_t*>(mx.p) + kMaxK * i);
      if (e != cudaSuccess) return cuda_fail(e, "load");
    }
    std::vector<uint32_t> hmx(kMaxK * std::max<uint32_t>(count, 1));
    cudaError_t e = cudaMemcpyAsync(hmx.data(), mx.p, 4 * hmx.size(), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "load maxima");
    cdl_status r = fetch(kSlotScratch, 1);
    if (r != CDL_OK) {
      cudaMemsetAsync(dslot(kSlotErr), 0, 8, st);
      return r;
    }
    for (uint32_t i = 0; i < count; ++i) {
      if (!ns[i]) continue;
      Relation& R = *rels[rl[i]];
      for (uint32_t k = 0; k < R.arity; ++k) R.bound[k] = std::max(R.bound[k], hmx[kMaxK * i + k]);
      R.pending.push_back(std::move(in[i]));
    }
    return CDL_OK;
  }

  // Sorts every relation's checked loads and merges them into its full
  // version (repeats dropped), all relations back to back with one read-back
  // of the sizes at the end.
  // Many relations of one arity loaded into empty relations are sorted and
  // deduplicated as one: a leading column numbers the relation of every
  // tuple, so one sort and one unique pass replace one of each per
  // relation, and the relations' rows are contiguous segments of the result.
  cdl_status flush_group(const std::vector<uint32_t>& grp, uint32_t k) {
    const uint32_t ng = (uint32_t)grp.size();
    std::vector<uint64_t> off{0};
    for (uint32_t i : grp) {
      uint64_t n = 0;
      for (const DCols& p : rels[i]->pending) n += p.n;
      off.push_back(off.back() + n);
    }
    const uint64_t N = off.back();
    if (N == 0 || N > 0xFFFFFFFFull) return CDL_OK;  // left to the relation-by-relation path
    DCols comb;
    DBuf doff = alloc(8 * off.size());
    if (!alloc_cols(comb, k + 1, N) || !doff.p) return fail(CDL_E_NOMEM, "grouped load");
    comb.n = N;
    cudaError_t e = cudaMemcpyAsync(doff.p, off.data(), 8 * off.size(), cudaMemcpyHostToDevice, st);
    for (uint32_t g = 0; g < ng && e == cudaSuccess; ++g) {
      uint64_t at = off[g];
      for (const DCols& p : rels[grp[g]]->pending) {
        for (uint32_t c = 0; c < k && e == cudaSuccess; ++c)
          e = cudaMemcpyAsync(comb.c[c + 1] + at, p.c[c], 4 * p.n, cudaMemcpyDeviceToDevice, st);
        at += p.n;
      }
    }
    if (e == cudaSuccess)
      e = fill_segments(ctx, comb.c[0], static_cast<const uint64_t*>(doff.p), ng, N);
    if (e != cudaSuccess) return cuda_fail(e, "grouped load");
    for (uint32_t i : grp) rels[i]->pending.clear();
    uint32_t bits[kMaxK] = {bits_of(ng - 1), 0, 0, 0};
    for (uint32_t i : grp)
      for (uint32_t c = 0; c < k; ++c) bits[c + 1] = std::max(bits[c + 1], bits_of(rels[i]->bound[c]));
    cdl_status r = sort_cols(comb, bits);
    if (r != CDL_OK) return r;
    DCols uniq;
    DBuf ws = alloc(diff_merge_workspace(0, N));
    if (!alloc_cols(uniq, k + 1, N) || !ws.p) return fail(CDL_E_NOMEM, "grouped load");
    e = diff_merge(ctx, k + 1, ColsIn{}, 0, comb.in(), N, uniq.out(), ColsOut{}, dslot(kSlotScratch),
                   ws.p);
    if (e != cudaSuccess) return cuda_fail(e, "grouped load");
    r = fetch(kSlotScratch, 1);
    if (r != CDL_OK) return r;
    const uint64_t nu = h_ctl[kSlotScratch];
    comb.clear();
    DBuf db = alloc(8 * (ng + 1));
    if (!db.p) return fail(CDL_E_NOMEM, "grouped load");
    std::vector<uint64_t> b(ng + 1);
    e = instance_bounds(ctx, uniq.c[0], nu, ng, static_cast<uint64_t*>(db.p));
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.data(), db.p, 8 * b.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "grouped load");
    for (uint32_t g = 0; g < ng; ++g) {
      Relation& R = *rels[grp[g]];
      const uint64_t cnt = b[g + 1] - b[g];
      if (!alloc_cols(R.full, k, std::max<uint64_t>(cnt, 1))) return fail(CDL_E_NOMEM, "grouped load");
      for (uint32_t c = 0; c < k && cnt; ++c) {
        e = cudaMemcpyAsync(R.full.c[c], uniq.c[c + 1] + b[g], 4 * cnt, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "grouped load");
      }
      R.full.n = cnt;
      R.version[kFull]++;
    }
    evict_stale();
    return CDL_OK;
  }

  cdl_status flush_loads() {
    for (uint32_t k = 1; k < (uint32_t)kMaxK; ++k) {  // groups of eight or more relations
      std::vector<uint32_t> grp;
      for (uint32_t i = 0; i < rels.size(); ++i) {
        const Relation& R = *rels[i];
        if (R.arity == k && !R.pending.empty() && R.full.n == 0) grp.push_back(i);
      }
      if (grp.size() < 8) continue;
      cdl_status r = flush_group(grp, k);
      if (r != CDL_OK) return r;
    }
    std::vector<uint32_t> done;
    for (uint32_t i = 0; i < rels.size(); ++i) {
      Relation& R = *rels[i];
      if (R.pending.empty()) continue;
      DCols in;
      if (R.pending.size() == 1) {
        in = std::move(R.pending[0]);
      } else {  // several loads: one buffer
        uint64_t n = 0;
        for (const DCols& p : R.pending) n += p.n;
        if (!alloc_cols(in, R.arity, n)) return fail(CDL_E_NOMEM, "load buffer");
        uint64_t at = 0;
        for (const DCols& p : R.pending) {
          for (uint32_t k = 0; k < R.arity; ++k) {
            cudaError_t e = cudaMemcpyAsync(in.c[k] + at, p.c[k], 4 * p.n, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "load copy");
          }
          at += p.n;
        }
        in.n = n;
      }
      R.pending.clear();
      uint32_t bits[kMaxK];
      for (uint32_t k = 0; k < R.arity; ++k) bits[k] = bits_of(R.bound[k]);
      cdl_status r = sort_cols(in, bits);
      if (r == CDL_OK) r = merge_into(R, in, nullptr, kSlotDelta + i);
      if (r != CDL_OK) return r;
      done.push_back(i);
    }
    if (done.empty()) return CDL_OK;
    cdl_status r = fetch(kSlotDelta, (uint32_t)rels.size());
    if (r != CDL_OK) return r;
    for (uint32_t i : done) rels[i]->full.n += h_ctl[kSlotDelta + i];
    evict_stale();
    return CDL_OK;
  }
};

// ------------------------------------------------------------------ C ABI

extern "C" {

void cdl_options_default(cdl_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->hash_load = 0.5;
  o->radix_bits = 0;
}

cdl_status cdl_create(const cdl_options* opts, cdl_engine** out) {
  if (!out) return CDL_E_INVALID;
  *out = nullptr;
  auto e = std::make_unique<cdl_engine>();
  if (opts) e->opt = *opts;
  else cdl_options_default(&e->opt);
  if (e->opt.dedup < 0 || e->opt.dedup > 2) return CDL_E_INVALID;
  e->st = static_cast<cudaStream_t>(e->opt.stream);
  e->pool.af = e->opt.alloc;
  e->pool.ff = e->opt.free;
  e->pool.ctx = e->opt.alloc_ctx;
  e->pool.limit = e->opt.mem_limit;
  e->hash_load = (e->opt.hash_load > 0 && e->opt.hash_load <= 0.9) ? e->opt.hash_load : 0.5;
  e->radix_bits = (e->opt.radix_bits >= 8 && e->opt.radix_bits <= 10) ? e->opt.radix_bits : 0;
  e->tuner.mode = e->opt.autotune < 0 ? 0 : (e->opt.autotune > 2 ? 2 : e->opt.autotune);
  e->tuner.path = e->opt.tune_cache ? e->opt.tune_cache : "";
  e->opt.tune_cache = nullptr;  // the engine keeps its own copy of the path
  if (e->tuner.mode) e->tuner.load();
  e->prof.on = e->opt.timing != 0;
  e->prof.mask = e->opt.timing == 1 ? ~0u : e->opt.timing >> 1;
  e->est_margin = e->opt.est_margin != 0.0 ? e->opt.est_margin : 1.0;
  if ((e->opt.alloc == nullptr) != (e->opt.free == nullptr)) return CDL_E_INVALID;
  e->ctl = e->alloc(kCtlSlots * sizeof(uint64_t));
  e->est_io = e->alloc(kEstFloats * sizeof(float));
  if (!e->ctl.p || !e->est_io.p) return CDL_E_NOMEM;
  if (cudaMallocHost(&e->h_ctl, kCtlSlots * sizeof(uint64_t)) != cudaSuccess ||
      cudaMallocHost(&e->h_est, kEstFloats * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return CDL_E_CUDA;
  }
  if (cudaMemsetAsync(e->ctl.p, 0, kCtlSlots * sizeof(uint64_t), e->st) != cudaSuccess)
    return CDL_E_CUDA;
  e->ctx.st = e->st;
  e->ctx.d_err = reinterpret_cast<uint32_t*>(e->dslot(kSlotErr));
  e->ctx.prof = &e->prof;
  if (e->opt.spin_limit) e->ctx.spin_limit = e->opt.spin_limit;
  *out = e.release();
  return CDL_OK;
}

cdl_status cdl_destroy(cdl_engine* e) {
  if (!e) return CDL_OK;
  cudaStreamSynchronize(e->st);
  delete e;
  return CDL_OK;
}

cdl_status cdl_relation_create(cdl_engine* e, const char* name, uint32_t arity, cdl_rel* out) {
  if (!e || !name || !out) return CDL_E_INVALID;
  if (e->ran) return e->fail(CDL_E_STATE, "relations must precede cdl_run");
  if (arity < 1 || arity > CDL_MAX_ARITY) return e->fail(CDL_E_INVALID, "arity must be 1..8");
  if (e->by_name.count(name)) return e->fail(CDL_E_INVALID, std::string("duplicate relation ") + name);
  if (e->rels.size() >= kMaxRels) return e->fail(CDL_E_INVALID, "too many relations");
  auto r = std::make_unique<Relation>();
  r->name = name;
  r->arity = arity;
  r->full.k = r->delta.k = r->fresh.k = arity;
  *out = (cdl_rel)e->rels.size();
  e->by_name[name] = *out;
  e->rels.push_back(std::move(r));
  return CDL_OK;
}

cdl_status cdl_relation_load(cdl_engine* e, cdl_rel rel, const uint32_t* const* cols, uint64_t n,
                             int on_device) {
  if (!e || (!cols && n)) return CDL_E_INVALID;
  if (rel >= e->rels.size()) return e->fail(CDL_E_INVALID, "no such relation");
  return e->load(rel, cols, n, on_device);
}

cdl_status cdl_relations_load(cdl_engine* e, uint32_t count, const cdl_rel* rels,
                              const uint32_t* const* const* cols, const uint64_t* n,
                              int on_device) {
  if (!e || (count && (!rels || !cols || !n))) return CDL_E_INVALID;
  return e->load_many(count, rels, cols, n, on_device);
}

cdl_status cdl_rule_add(cdl_engine* e, const cdl_rule* rule) {
  if (!e || !rule) return CDL_E_INVALID;
  if (e->ran) return e->fail(CDL_E_STATE, "rules must precede cdl_run");
  if (rule->nbody < 1 || rule->nbody > CDL_MAX_BODY || !rule->body)
    return e->fail(CDL_E_INVALID, "a rule needs 1..8 body atoms");
  auto conv = [&](const cdl_atom& a, AtomR& out) -> bool {
    if (a.rel >= e->rels.size() || a.arity != e->rels[a.rel]->arity || !a.terms) return false;
    out.rel = a.rel;
    for (uint32_t k = 0; k < a.arity; ++k) {
      if (a.terms[k].is_const && a.terms[k].v == CDL_EMPTY_KEY) return false;
      out.t.push_back(Term{a.terms[k].is_const != 0, a.terms[k].v});
    }
    return true;
  };
  RuleR r;
  if (!conv(rule->head, r.head)) return e->fail(CDL_E_INVALID, "bad head atom");
  std::vector<uint32_t> body_vars;
  for (uint32_t i = 0; i < rule->nbody; ++i) {
    AtomR a;
    if (!conv(rule->body[i], a)) return e->fail(CDL_E_INVALID, "bad body atom");
    for (const Term& t : a.t)
      if (!t.is_const) body_vars.push_back(t.v);
    r.body.push_back(a);
  }
  auto bound = [&](uint32_t v) {
    return std::find(body_vars.begin(), body_vars.end(), v) != body_vars.end();
  };
  for (const Term& t : r.head.t)
    if (!t.is_const && !bound(t.v)) return e->fail(CDL_E_INVALID, "head variable not in body");
  if (rule->nneq > 4 || (rule->nneq && !rule->neq)) return e->fail(CDL_E_INVALID, "bad inequalities");
  for (uint32_t i = 0; i < rule->nneq; ++i) {
    const uint32_t a = rule->neq[2 * i], b = rule->neq[2 * i + 1];
    if (!bound(a) || !bound(b)) return e->fail(CDL_E_INVALID, "inequality variable not in body");
    r.neq.emplace_back(a, b);
  }
  e->rules.push_back(std::move(r));
  return CDL_OK;
}

cdl_status cdl_run(cdl_engine* e, cdl_stats* stats) {
  if (!e) return CDL_E_INVALID;
  return e->run(stats);
}

cdl_status cdl_relation_size(cdl_engine* e, cdl_rel rel, uint64_t* n) {
  if (!e || !n) return CDL_E_INVALID;
  if (rel >= e->rels.size()) return e->fail(CDL_E_INVALID, "no such relation");
  const cdl_status f = e->flush_loads();
  if (f != CDL_OK) return f;
  *n = e->rels[rel]->full.n;
  return CDL_OK;
}

cdl_status cdl_relation_export(cdl_engine* e, cdl_rel rel, uint32_t* const* cols, uint64_t cap,
                               uint64_t* n_written, int on_device) {
  if (!e || !n_written) return CDL_E_INVALID;
  if (rel >= e->rels.size()) return e->fail(CDL_E_INVALID, "no such relation");
  const cdl_status f = e->flush_loads();
  if (f != CDL_OK) return f;
  const Relation& R = *e->rels[rel];
  (void)on_device;  // the copies infer both sides' memory (Full may be host-resident)
  *n_written = R.full.n;
  if (cap < R.full.n) return e->fail(CDL_E_CAPACITY, "export buffer too small");
  if (R.full.n == 0) return CDL_OK;
  if (!cols) return CDL_E_INVALID;
  cudaError_t er = cudaSuccess;
  for (uint32_t k = 0; k < R.arity && er == cudaSuccess; ++k) {
    if (!cols[k]) return e->fail(CDL_E_INVALID, "null column pointer");
    // Full may be in device or (option host_full) pinned host memory
    er = cudaMemcpyAsync(cols[k], R.full.c[k], R.full.n * 4, cudaMemcpyDefault, e->st);
  }
  if (er == cudaSuccess) er = cudaStreamSynchronize(e->st);
  return er == cudaSuccess ? CDL_OK : e->cuda_fail(er, "export");
}

cdl_status cdl_checkpoint_save(cdl_engine* e, const char* path) {
  return e ? e->checkpoint_save(path) : CDL_E_INVALID;
}

cdl_status cdl_checkpoint_load(cdl_engine* e, const char* path) {
  return e ? e->checkpoint_load(path) : CDL_E_INVALID;
}

cdl_status cdl_relation_export_rows(cdl_engine* e, cdl_rel rel, uint64_t first, uint64_t count,
                                    uint32_t* const* cols, int on_device) {
  if (!e) return CDL_E_INVALID;
  if (rel >= e->rels.size()) return e->fail(CDL_E_INVALID, "no such relation");
  const cdl_status f = e->flush_loads();
  if (f != CDL_OK) return f;
  const Relation& R = *e->rels[rel];
  (void)on_device;  // the copies infer both sides' memory (Full may be host-resident)
  if (first > R.full.n || count > R.full.n - first)
    return e->fail(CDL_E_CAPACITY, "row range past the relation");
  if (count == 0) return CDL_OK;
  if (!cols) return CDL_E_INVALID;
  cudaError_t er = cudaSuccess;
  for (uint32_t k = 0; k < R.arity && er == cudaSuccess; ++k) {
    if (!cols[k]) return e->fail(CDL_E_INVALID, "null column pointer");
    er = cudaMemcpyAsync(cols[k], R.full.c[k] + first, count * 4, cudaMemcpyDefault, e->st);
  }
  if (er == cudaSuccess) er = cudaStreamSynchronize(e->st);
  return er == cudaSuccess ? CDL_OK : e->cuda_fail(er, "export rows");
}

cdl_status cdl_instance_rows(cdl_engine* e, cdl_rel rel, uint32_t instance, uint64_t* first,
                             uint64_t* count) {
  if (!e || !first || !count) return CDL_E_INVALID;
  if (rel >= e->rels.size()) return e->fail(CDL_E_INVALID, "no such relation");
  if (!e->opt.n_instances || instance >= e->opt.n_instances)
    return e->fail(CDL_E_INVALID, "no such instance");
  const Relation& R = *e->rels[rel];
  *first = *count = 0;
  if (R.full.n == 0) return CDL_OK;
  DBuf b = e->alloc(8 * (e->opt.n_instances + 1));
  if (!b.p) return e->fail(CDL_E_NOMEM, "instance bounds");
  uint64_t* d = static_cast<uint64_t*>(b.p);
  uint64_t h[2] = {0, 0};
  cudaError_t er = instance_bounds(e->ctx, R.full.c[0], R.full.n, e->opt.n_instances, d);
  if (er == cudaSuccess) er = cudaMemcpyAsync(h, d + instance, 16, cudaMemcpyDeviceToHost, e->st);
  if (er == cudaSuccess) er = cudaStreamSynchronize(e->st);
  if (er != cudaSuccess) return e->cuda_fail(er, "instance bounds");
  *first = h[0];
  *count = h[1] - h[0];
  return CDL_OK;
}

cdl_status cdl_kernel_profile(cdl_engine* e, uint32_t idx, char* name, size_t name_cap,
                              uint64_t* launches, double* ms, double* bytes) {
  if (!e) return CDL_E_INVALID;
  if (idx >= (uint32_t)kNumClasses) return CDL_E_INVALID;
  if (name && name_cap) {
    std::strncpy(name, kernel_class_name((int)idx), name_cap - 1);
    name[name_cap - 1] = 0;
  }
  if (launches) *launches = e->prof.launches[idx];
  if (ms) *ms = e->prof.ms[idx];
  if (bytes) *bytes = e->prof.bytes[idx];
  return CDL_OK;
}

const char* cdl_last_error(const cdl_engine* e) { return e ? e->err.c_str() : "no engine"; }

cdl_status cdl_estimator_log(cdl_engine* e, float* X, float* y, uint64_t cap, uint64_t* n) {
  if (!e || !n) return CDL_E_INVALID;
  *n = e->log_y.size();
  const uint64_t m = std::min<uint64_t>(cap, *n);
  if (X) std::memcpy(X, e->log_x.data(), sizeof(float) * kMlpIn * m);
  if (y) std::memcpy(y, e->log_y.data(), sizeof(float) * m);
  return CDL_OK;
}

cdl_status cdl_estimator_train(cdl_engine* e, const float* X, const float* y, uint64_t n,
                               uint32_t epochs, float lr, float tau, uint64_t seed, float* loss) {
  if (!e || !(tau > 0.f && tau < 1.f) || !(lr > 0.f)) return CDL_E_INVALID;
  return e->train(X, y, n, epochs, lr, tau, seed, loss);
}

cdl_status cdl_estimator_params(cdl_engine* e, float* params, int set) {
  if (!e || !params) return CDL_E_INVALID;
  if (set) return e->install_weights(params);
  if (!e->est_weights) return e->fail(CDL_E_STATE, "no trained estimator");
  cudaError_t er = cudaMemcpyAsync(params, e->est_w.p, sizeof(float) * kMlpParams,
                                   cudaMemcpyDeviceToHost, e->st);
  if (er == cudaSuccess) er = cudaStreamSynchronize(e->st);
  return er == cudaSuccess ? CDL_OK : e->cuda_fail(er, "estimator params");
}

}  // extern "C"
