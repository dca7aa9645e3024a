// Autotuner of the engine's launch parameters: radix digit width and block
// size of the sort passes, hash-table load factor of the join indexes.
//
// A decision has a key (the parameter and the size class it is taken for)
// and a few candidates.  In tuning mode every candidate is first measured
// kTrials times; afterwards, and in cache mode, the candidate with the
// lowest mean cost wins (the engine's configured value until one is
// measured).  Costs are device nanoseconds per element, read from CUDA
// events recorded around the launches the decision shapes; results persist
// in a text file, one "key candidate trials summed_cost" line per entry.
// No choice changes a result: every candidate computes the same tuples.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

namespace cdl {

struct Tuner {
  static constexpr uint32_t kTrials = 2;
  int mode = 0;  // 0 off, 1 use the cache file, 2 measure untried candidates
  std::string path;
  bool dirty = false;
  struct Stat {
    uint32_t n = 0;
    double sum = 0;
  };
  std::map<std::string, std::vector<Stat>> table;
  struct Probe {
    int idx = -1;  // pending measurement, -1 when none
  };
  struct Pending {
    std::string key;
    int cand;
    double units;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> events;

  // The candidate to use for key among ncand (0 = the configured default).
  int choose(const std::string& key, int ncand, bool* measuring);
  // Brackets the launches of one decision on stream st; units = elements.
  Probe start(const std::string& key, int cand, double units, cudaStream_t st);
  void stop(const Probe& p, cudaStream_t st);
  // Folds finished measurements into the table (call after a sync).
  void resolve();
  bool load();
  bool save();
  ~Tuner();
};

}  // namespace cdl
