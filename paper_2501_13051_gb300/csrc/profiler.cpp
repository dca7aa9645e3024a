// CUDA-event timing of kernel classes (engine option `timing`).
#include "kernels.h"

namespace cdl {

const char* kernel_class_name(int c) {
  static const char* names[kNumClasses] = {
      "hash_build", "count_heads", "join_count", "scan",      "join_write", "radix_upsweep",
      "radix_scatter", "diff_count", "diff_merge", "select", "misc",
      "estimator", "join_direct", "retire", "dense", "dedup"};
  return (c >= 0 && c < kNumClasses) ? names[c] : "?";
}

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Profiler::begin(int cls, cudaStream_t st) {
  ++total_launches;
  if (!on || !(mask >> cls & 1u)) return;
  Rec r{cls, get(), get(), 0.0};
  cudaEventRecord(r.a, st);
  open.push_back(r);
}

void Profiler::end(int cls, double algo_bytes, cudaStream_t st) {
  total_bytes += algo_bytes;
  if (!on || !(mask >> cls & 1u)) return;
  for (auto it = open.rbegin(); it != open.rend(); ++it) {
    if (it->cls == cls && it->bytes == 0.0) {
      cudaEventRecord(it->b, st);
      it->bytes = algo_bytes > 0 ? algo_bytes : 1e-30;
      return;
    }
  }
}

void Profiler::add_bytes(int cls, double b) {
  total_bytes += b;
  if (!on || !(mask >> cls & 1u)) return;
  for (auto it = open.rbegin(); it != open.rend(); ++it) {
    if (it->cls == cls) {
      it->bytes += b;
      return;
    }
  }
}

void Profiler::collect() {
  for (Rec& r : open) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      launches[r.cls] += 1;
      ms[r.cls] += t;
      bytes[r.cls] += r.bytes > 1e-20 ? r.bytes : 0.0;
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  open.clear();
}

void Profiler::reset() {
  collect();
  for (int i = 0; i < kNumClasses; ++i) {
    launches[i] = 0;
    ms[i] = 0;
    bytes[i] = 0;
  }
  total_launches = 0;
  total_bytes = 0;
}

Profiler::~Profiler() {
  for (Rec& r : open) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

}  // namespace cdl
