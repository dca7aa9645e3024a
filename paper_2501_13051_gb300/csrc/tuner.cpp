// Autotuner bookkeeping (see tuner.h).
#include "tuner.h"

#include <cstdio>

namespace cdl {

int Tuner::choose(const std::string& key, int ncand, bool* measuring) {
  *measuring = false;
  if (mode == 0 || ncand <= 1) return 0;
  std::vector<Stat>& s = table[key];
  if (s.size() < (size_t)ncand) s.resize(ncand);
  if (mode == 2)
    for (int c = 0; c < ncand; ++c)
      if (s[c].n < kTrials) {
        *measuring = true;
        return c;
      }
  int best = 0;
  double best_cost = -1;
  for (int c = 0; c < ncand; ++c) {
    if (!s[c].n) continue;
    const double m = s[c].sum / s[c].n;
    if (best_cost < 0 || m < best_cost) {
      best_cost = m;
      best = c;
    }
  }
  return best;
}

Tuner::Probe Tuner::start(const std::string& key, int cand, double units, cudaStream_t st) {
  Probe p;
  if (mode != 2 || units <= 0) return p;
  cudaEvent_t ev[2];
  for (cudaEvent_t& e : ev) {
    if (!events.empty()) {
      e = events.back();
      events.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
      return p;
    }
  }
  cudaEventRecord(ev[0], st);
  pending.push_back(Pending{key, cand, units, ev[0], ev[1]});
  p.idx = (int)pending.size() - 1;
  return p;
}

void Tuner::stop(const Probe& p, cudaStream_t st) {
  if (p.idx >= 0) cudaEventRecord(pending[p.idx].b, st);
}

void Tuner::resolve() {
  for (Pending& q : pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(q.b) == cudaSuccess &&
        cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      std::vector<Stat>& s = table[q.key];
      if (s.size() <= (size_t)q.cand) s.resize(q.cand + 1);
      s[q.cand].n += 1;
      s[q.cand].sum += 1e6 * ms / q.units;
      dirty = true;
    }
    events.push_back(q.a);
    events.push_back(q.b);
  }
  pending.clear();
}

bool Tuner::load() {
  if (path.empty()) return true;
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return true;  // nothing tuned yet
  char key[256];
  int cand = 0;
  unsigned n = 0;
  double sum = 0;
  while (std::fscanf(f, "%255s %d %u %lf", key, &cand, &n, &sum) == 4) {
    if (cand < 0 || cand > 64) continue;
    std::vector<Stat>& s = table[key];
    if (s.size() <= (size_t)cand) s.resize(cand + 1);
    s[cand].n = n;
    s[cand].sum = sum;
  }
  std::fclose(f);
  return true;
}

bool Tuner::save() {
  if (path.empty() || !dirty) return true;
  FILE* f = std::fopen(path.c_str(), "w");
  if (!f) return false;
  for (const auto& kv : table)
    for (size_t c = 0; c < kv.second.size(); ++c)
      if (kv.second[c].n)
        std::fprintf(f, "%s %zu %u %.6f\n", kv.first.c_str(), c, kv.second[c].n, kv.second[c].sum);
  std::fclose(f);
  dirty = false;
  return true;
}

Tuner::~Tuner() {
  for (Pending& q : pending) {
    cudaEventDestroy(q.a);
    cudaEventDestroy(q.b);
  }
  for (cudaEvent_t e : events) cudaEventDestroy(e);
}

}  // namespace cdl
