// C ABI of the single steps (include/cdl.h, "Steps of one round"): the
// engine's own kernels on caller-owned device buffers, scratch carved from a
// caller-provided workspace.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/cdl.h"
#include "kernels.h"

using namespace cdl;

namespace {

size_t up(size_t b) { return (b + 255) & ~size_t(255); }

// Carves consecutive 256-byte aligned pieces out of a workspace.
struct Carve {
  char* p;
  size_t used = 0;
  explicit Carve(void* base) : p(static_cast<char*>(base)) {}
  void* take(size_t b) {
    void* r = p ? p + used : nullptr;
    used += up(b);
    return r;
  }
};

constexpr size_t kHead = 256;  // error word, cursor, totals

bool pow2(uint64_t x) { return x && !(x & (x - 1)); }

cdl_status cuda_status(cudaError_t e) { return e == cudaSuccess ? CDL_OK : CDL_E_CUDA; }

cdl_status read_flags(uint64_t* head, cudaStream_t st, uint64_t* host, int n) {
  if (cudaMemcpyAsync(host, head, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CDL_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CDL_E_CUDA;
  const uint32_t f = (uint32_t)host[0];
  if (f & kErrTimeout) return CDL_E_TIMEOUT;
  if (f & kErrCapacity) return CDL_E_CAPACITY;
  if (f & kErrTable) return CDL_E_CAPACITY;
  if (f & kErrValue) return CDL_E_VALUE;
  return CDL_OK;
}

uint32_t bits_of(uint32_t v) {
  uint32_t b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

}  // namespace

extern "C" {

uint64_t cdl_hash_table_bytes(uint64_t n_keys, double load) {
  return table_slots(n_keys, load) * sizeof(Slot);
}

cdl_status cdl_hash_build(const uint32_t* keys, uint64_t n, void* table, uint64_t table_bytes,
                          void* stream) {
  if ((!keys && n) || !table) return CDL_E_INVALID;
  const uint64_t slots = table_bytes / sizeof(Slot);
  if (!pow2(slots) || slots <= n) return CDL_E_INVALID;
  if (n > 0xFFFFFFFFull) return CDL_E_CAPACITY;
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  return cuda_status(hash_build(c, keys, nullptr, n, static_cast<Slot*>(table), slots));
}

cdl_status cdl_join_count(const uint32_t* probe, uint64_t n, const void* table,
                          uint64_t table_bytes, uint32_t* counts, void* stream) {
  if ((!probe || !counts) && n) return CDL_E_INVALID;
  const uint64_t slots = table_bytes / sizeof(Slot);
  if (!table || !pow2(slots)) return CDL_E_INVALID;
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  JoinSpec j{};
  j.probe.c[0] = probe;
  j.n_probe = n;
  j.pk0 = 0;
  j.pk1 = 0xFFu;
  j.table = static_cast<const Slot*>(table);
  j.slots = slots;
  return cuda_status(join_count_only(c, j, counts));
}

cdl_status cdl_exclusive_scan(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* total_host,
                              void* workspace, size_t* ws_bytes, void* stream) {
  if (!ws_bytes) return CDL_E_INVALID;
  const size_t need = kHead + up(scan_workspace(n));
  if (!workspace) {
    *ws_bytes = need;
    return CDL_OK;
  }
  if (*ws_bytes < need || ((!in || !out) && n)) return CDL_E_INVALID;
  Carve cv(workspace);
  uint64_t* head = static_cast<uint64_t*>(cv.take(kHead));
  void* sws = cv.take(scan_workspace(n));
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(head, 0, kHead, c.st);
  if (e == cudaSuccess) e = exclusive_scan(c, in, n, out, head + 1, sws);
  if (e != cudaSuccess) return CDL_E_CUDA;
  if (total_host) {
    uint64_t h[2];
    cdl_status s = read_flags(head, c.st, h, 2);
    if (s != CDL_OK) return s;
    *total_host = h[1];
  }
  return CDL_OK;
}

cdl_status cdl_join(const uint32_t* const* probe_cols, uint32_t probe_arity, uint64_t n_probe,
                    uint32_t probe_key, const uint32_t* const* build_cols, uint32_t build_arity,
                    uint64_t n_build, uint32_t build_key, const cdl_colref* spec,
                    uint32_t out_arity, const cdl_colref* neq, uint32_t nneq,
                    uint32_t* const* out_cols, uint64_t out_cap, uint64_t* n_out, void* workspace,
                    size_t* ws_bytes, void* stream) {
  if (!ws_bytes) return CDL_E_INVALID;
  const uint64_t slots = table_slots(n_build, 0.5);
  const size_t need = kHead + up(slots * sizeof(Slot)) + up(8 * (n_probe ? n_probe : 1)) +
                      up(join_count_workspace(n_probe));
  if (!workspace) {
    *ws_bytes = need;
    return CDL_OK;
  }
  if (*ws_bytes < need || !n_out) return CDL_E_INVALID;
  if (probe_arity < 1 || probe_arity > CDL_MAX_ARITY || build_arity < 1 ||
      build_arity > CDL_MAX_ARITY || out_arity < 1 || out_arity > CDL_MAX_ARITY ||
      probe_key >= probe_arity || build_key >= build_arity || nneq > 4 || !spec)
    return CDL_E_INVALID;
  if (n_build > 0xFFFFFFFFull) return CDL_E_CAPACITY;
  JoinSpec j{};
  for (uint32_t k = 0; k < probe_arity; ++k) j.probe.c[k] = probe_cols[k];
  for (uint32_t k = 0; k < build_arity; ++k) j.build.c[k] = build_cols[k];
  j.n_probe = n_probe;
  j.pk0 = probe_key;
  j.pk1 = 0xFFu;
  auto conv = [&](const cdl_colref& r, Ref& out) {
    if (r.side > 2) return false;
    if (r.side == 0 && r.v >= probe_arity) return false;
    if (r.side == 1 && r.v >= build_arity) return false;
    out = Ref{(uint8_t)r.side, r.v};
    return true;
  };
  j.out_k = out_arity;
  for (uint32_t k = 0; k < out_arity; ++k)
    if (!conv(spec[k], j.out[k])) return CDL_E_INVALID;
  j.n_neq = nneq;
  for (uint32_t q = 0; q < nneq; ++q)
    if (!conv(neq[2 * q], j.neq[q][0]) || !conv(neq[2 * q + 1], j.neq[q][1])) return CDL_E_INVALID;
  Carve cv(workspace);
  uint64_t* head = static_cast<uint64_t*>(cv.take(kHead));
  Slot* table = static_cast<Slot*>(cv.take(slots * sizeof(Slot)));
  uint64_t* off = static_cast<uint64_t*>(cv.take(8 * (n_probe ? n_probe : 1)));
  void* cws = cv.take(join_count_workspace(n_probe));
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  c.d_err = reinterpret_cast<uint32_t*>(head);
  cudaError_t e = cudaMemsetAsync(head, 0, kHead, c.st);
  if (e == cudaSuccess) e = hash_build(c, build_cols[build_key], nullptr, n_build, table, slots);
  j.table = table;
  j.slots = slots;
  if (e == cudaSuccess) e = join_count_scan(c, j, off, head + 1, cws);
  if (e != cudaSuccess) return CDL_E_CUDA;
  uint64_t h[3];
  cdl_status s = read_flags(head, c.st, h, 2);
  if (s != CDL_OK) return s;
  const uint64_t total = h[1];
  *n_out = total;
  if (total == 0) return CDL_OK;
  if (out_cap < total) return CDL_E_CAPACITY;
  ColsOut out;
  for (uint32_t k = 0; k < CDL_MAX_ARITY; ++k) out.c[k] = k < out_arity ? out_cols[k] : nullptr;
  // the count workspace is free again: it holds the write splits if large enough
  e = join_write(c, j, off, total, out, 0, head + 2, out_cap, cws, join_count_workspace(n_probe));
  if (e != cudaSuccess) return CDL_E_CUDA;
  s = read_flags(head, c.st, h, 3);
  if (s != CDL_OK) return s;
  *n_out = h[2];
  return CDL_OK;
}

cdl_status cdl_sort_unique(const uint32_t* const* cols, uint32_t arity, uint64_t n,
                           uint32_t* const* out_cols, uint64_t* n_out, void* workspace,
                           size_t* ws_bytes, void* stream) {
  if (!ws_bytes || arity < 1 || arity > CDL_MAX_ARITY) return CDL_E_INVALID;
  const uint64_t rows = n ? n : 1;
  const size_t col = up(rows * 4);
  const size_t need = kHead + 2 * arity * col + up(radix_workspace(n, 9)) +
                      up(diff_merge_workspace(0, n));
  if (!workspace) {
    *ws_bytes = need;
    return CDL_OK;
  }
  if (*ws_bytes < need || !n_out || ((!cols || !out_cols) && n)) return CDL_E_INVALID;
  if (n > 0xFFFFFFFFull) return CDL_E_CAPACITY;
  Carve cv(workspace);
  uint64_t* head = static_cast<uint64_t*>(cv.take(kHead));
  ColsOut a{}, b{};
  for (uint32_t k = 0; k < arity; ++k) a.c[k] = static_cast<uint32_t*>(cv.take(rows * 4));
  for (uint32_t k = 0; k < arity; ++k) b.c[k] = static_cast<uint32_t*>(cv.take(rows * 4));
  void* rws = cv.take(radix_workspace(n, 9));  // room for 9-bit digits
  void* dws = cv.take(diff_merge_workspace(0, n));
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  c.d_err = reinterpret_cast<uint32_t*>(head);
  cudaError_t e = cudaMemsetAsync(head, 0, kHead, c.st);
  for (uint32_t k = 0; k < arity && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(a.c[k], cols[k], n * 4, cudaMemcpyDeviceToDevice, c.st);
  ColsIn ain;
  for (int k = 0; k < kMaxK; ++k) ain.c[k] = a.c[k];
  uint32_t* dmax = reinterpret_cast<uint32_t*>(head + 4);
  if (e == cudaSuccess) e = column_max(c, ain, arity, n, dmax);
  if (e != cudaSuccess) return CDL_E_CUDA;
  uint64_t h[8];
  cdl_status s = read_flags(head, c.st, h, 6);
  if (s != CDL_OK) return s;
  uint32_t bits[kMaxK] = {0, 0, 0, 0};
  const uint32_t* hm = reinterpret_cast<const uint32_t*>(h + 4);
  for (uint32_t k = 0; k < arity; ++k) bits[k] = bits_of(hm[k]);
  uint32_t total = 0;
  for (uint32_t k = 0; k < arity; ++k) total += bits[k];
  RadixPlan plan = make_radix_plan(arity, bits, fit_digit_bits(total, 8));
  bool in_b = false;
  e = radix_sort(c, plan, a, b, n, rws, &in_b);
  if (e != cudaSuccess) return CDL_E_CUDA;
  ColsIn sorted;
  for (int k = 0; k < kMaxK; ++k) sorted.c[k] = in_b ? b.c[k] : a.c[k];
  ColsOut delta{}, none{};
  for (uint32_t k = 0; k < arity; ++k) delta.c[k] = out_cols[k];
  ColsIn empty{};
  e = diff_merge(c, arity, empty, 0, sorted, n, delta, none, head + 1, dws);
  if (e != cudaSuccess) return CDL_E_CUDA;
  s = read_flags(head, c.st, h, 2);
  if (s != CDL_OK) return s;
  *n_out = h[1];
  return CDL_OK;
}

cdl_status cdl_mlp_forward(const float* params, const float* X, uint64_t n, float* out,
                           void* workspace, size_t* ws_bytes, void* stream) {
  if (!ws_bytes) return CDL_E_INVALID;
  const size_t need = mlp_workspace(n);
  if (!workspace) {
    *ws_bytes = need;
    return CDL_OK;
  }
  if (*ws_bytes < need || !params || ((!X || !out) && n)) return CDL_E_INVALID;
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  return cuda_status(mlp_forward(c, params, X, n, out, workspace));
}

cdl_status cdl_mlp_gradient(const float* params, const float* X, const float* y, uint64_t n,
                            float tau, float* out, float* grad, void* workspace, size_t* ws_bytes,
                            void* stream) {
  if (!ws_bytes) return CDL_E_INVALID;
  const size_t need = mlp_workspace(n);
  if (!workspace) {
    *ws_bytes = need;
    return CDL_OK;
  }
  if (*ws_bytes < need || !params || !grad || ((!X || !y || !out) && n)) return CDL_E_INVALID;
  if (!(tau > 0.f && tau < 1.f)) return CDL_E_INVALID;
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  return cuda_status(mlp_gradient(c, params, X, y, n, tau, out, grad, workspace));
}

cdl_status cdl_mlp_infer_bf16(const float* params, const float* X, uint64_t n, float* out,
                              void* workspace, size_t* ws_bytes, void* stream) {
  if (!ws_bytes) return CDL_E_INVALID;
  const size_t need = up(sizeof(uint16_t) * kMlpParams);
  if (!workspace) {
    *ws_bytes = need;
    return CDL_OK;
  }
  if (*ws_bytes < need || !params || ((!X || !out) && n)) return CDL_E_INVALID;
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  cudaError_t e = mlp_to_bf16(c, params, workspace);
  if (e == cudaSuccess) e = mlp_infer_bf16(c, workspace, X, n, out);
  return cuda_status(e);
}

cdl_status cdl_mlp_adam(float* params, const float* grad, float* m, float* v, uint64_t step,
                        float lr, void* stream) {
  if (!params || !grad || !m || !v || step == 0) return CDL_E_INVALID;
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  return cuda_status(mlp_adam(c, params, grad, m, v, step, lr));
}

cdl_status cdl_join_features(const uint32_t* probe_k0, const uint32_t* probe_k1, uint64_t n_probe,
                             const uint32_t* build_k0, const uint32_t* build_k1, uint64_t n_build,
                             const float* host, float* features, void* stream) {
  if (!host || !features || (n_probe && !probe_k0) || (n_build && !build_k0)) return CDL_E_INVALID;
  JoinFeatureHost hf{host[0], host[1], host[2], host[3], host[4], host[5]};
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  return cuda_status(join_features(c, probe_k0, probe_k1, n_probe, build_k0, build_k1, n_build,
                                   hf, features));
}

cdl_status cdl_diff_merge(const uint32_t* const* full, uint64_t n_full,
                          const uint32_t* const* fresh, uint64_t n_fresh, uint32_t arity,
                          uint32_t* const* delta, uint64_t* n_delta, uint32_t* const* merged,
                          void* workspace, size_t* ws_bytes, void* stream) {
  if (!ws_bytes || arity < 1 || arity > CDL_MAX_ARITY) return CDL_E_INVALID;
  const size_t need = kHead + up(diff_merge_workspace(n_full, n_fresh));
  if (!workspace) {
    *ws_bytes = need;
    return CDL_OK;
  }
  if (*ws_bytes < need || !n_delta) return CDL_E_INVALID;
  if ((n_full && !full) || (n_fresh && !fresh) || !delta || !merged) return CDL_E_INVALID;
  Carve cv(workspace);
  uint64_t* head = static_cast<uint64_t*>(cv.take(kHead));
  void* dws = cv.take(diff_merge_workspace(n_full, n_fresh));
  ColsIn f{}, u{};
  ColsOut d{}, m{};
  for (uint32_t k = 0; k < arity; ++k) {
    f.c[k] = n_full ? full[k] : nullptr;
    u.c[k] = n_fresh ? fresh[k] : nullptr;
    d.c[k] = delta[k];
    m.c[k] = merged[k];
  }
  Ctx c;
  c.st = static_cast<cudaStream_t>(stream);
  c.d_err = reinterpret_cast<uint32_t*>(head);
  cudaError_t e = cudaMemsetAsync(head, 0, kHead, c.st);
  if (e == cudaSuccess) e = diff_merge(c, arity, f, n_full, u, n_fresh, d, m, head + 1, dws);
  if (e != cudaSuccess) return CDL_E_CUDA;
  uint64_t h[2];
  cdl_status s = read_flags(head, c.st, h, 2);
  if (s != CDL_OK) return s;
  *n_delta = h[1];
  return CDL_OK;
}

}  // extern "C"
