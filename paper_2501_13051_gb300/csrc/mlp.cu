// The learned join-size estimator (an addition of this library; the paper
// sizes every join exactly, Algorithm 1's count pass).  A 16 -> 64 -> 64 -> 1
// ReLU network predicts log2(1 + join output size) from 16 features of the
// join; the engine sizes the output buffer from the prediction, writes the
// join in a single pass, and falls back to the exact three-pass join when
// the prediction was too small.  Tuple results never depend on the network.
//
// Training runs in FP32 on these kernels: forward per sample (one block of
// 64 threads), backward of the activations per sample, then every parameter
// gradient as a sum over the batch computed by one thread per parameter
// (deterministic: no atomics), pinball (quantile) loss at level tau, Adam
// update (Kingma & Ba, 2015).  Inference runs with BF16 weights and
// activations and FP32 accumulation.
//
// Parameters: one flat FP32 vector W1 (64x16 row-major), b1, W2 (64x64
// row-major), b2, w3 (64), b3: 5313 values.
#include <cuda_bf16.h>

#include <cmath>

#include "kernels.h"

namespace cdl {

namespace {

constexpr int kIn = kMlpIn, kH = kMlpHidden;
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, ow3 = ob2 + kH,
              ob3 = ow3 + kH;
static_assert(ob3 + 1 == kMlpParams, "parameter layout");

__device__ __forceinline__ float block64_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  const float s = red[0] + red[1];
  __syncthreads();
  return s;
}

// Z1, Z2: pre-activations (n x 64); out: prediction per sample.
__global__ void __launch_bounds__(kH) k_mlp_forward(const float* __restrict__ th,
                                                    const float* __restrict__ X, uint64_t n,
                                                    float* __restrict__ Z1, float* __restrict__ Z2,
                                                    float* __restrict__ out) {
  __shared__ float x[kIn], h1[kH], red[2];
  const uint64_t s = blockIdx.x;
  const int t = threadIdx.x;
  if (t < kIn) x[t] = X[s * kIn + t];
  __syncthreads();
  float z1 = th[ob1 + t];
#pragma unroll
  for (int k = 0; k < kIn; ++k) z1 += th[oW1 + t * kIn + k] * x[k];
  Z1[s * kH + t] = z1;
  h1[t] = fmaxf(z1, 0.f);
  __syncthreads();
  float z2 = th[ob2 + t];
#pragma unroll 16
  for (int i = 0; i < kH; ++i) z2 += th[oW2 + t * kH + i] * h1[i];
  Z2[s * kH + t] = z2;
  const float o = block64_sum(th[ow3 + t] * fmaxf(z2, 0.f), red);
  if (t == 0) out[s] = o + th[ob3];
}

// Per sample: GO = dL/dprediction, G2 = dL/dZ2, G1 = dL/dZ1.
__global__ void __launch_bounds__(kH) k_mlp_backward(const float* __restrict__ th,
                                                     const float* __restrict__ y, uint64_t n,
                                                     float tau, const float* __restrict__ Z1,
                                                     const float* __restrict__ Z2,
                                                     const float* __restrict__ out,
                                                     float* __restrict__ GO, float* __restrict__ G1,
                                                     float* __restrict__ G2) {
  __shared__ float g2[kH];
  const uint64_t s = blockIdx.x;
  const int t = threadIdx.x;
  const float g = (y[s] > out[s] ? -tau : 1.f - tau) / (float)n;
  if (t == 0) GO[s] = g;
  const float gz2 = Z2[s * kH + t] > 0.f ? g * th[ow3 + t] : 0.f;
  G2[s * kH + t] = gz2;
  g2[t] = gz2;
  __syncthreads();
  float a = 0.f;
#pragma unroll 16
  for (int j = 0; j < kH; ++j) a += g2[j] * th[oW2 + j * kH + t];
  G1[s * kH + t] = Z1[s * kH + t] > 0.f ? a : 0.f;
}

// One thread per parameter: its gradient summed over the batch in order.
__global__ void k_mlp_param_grads(const float* __restrict__ X, uint64_t n,
                                  const float* __restrict__ Z1, const float* __restrict__ Z2,
                                  const float* __restrict__ GO, const float* __restrict__ G1,
                                  const float* __restrict__ G2, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  float acc = 0.f;
  if (p < ob1) {
    const int i = p / kIn, k = p % kIn;
    for (uint64_t s = 0; s < n; ++s) acc += G1[s * kH + i] * X[s * kIn + k];
  } else if (p < oW2) {
    const int i = p - ob1;
    for (uint64_t s = 0; s < n; ++s) acc += G1[s * kH + i];
  } else if (p < ob2) {
    const int j = (p - oW2) / kH, i = (p - oW2) % kH;
    for (uint64_t s = 0; s < n; ++s) acc += G2[s * kH + j] * fmaxf(Z1[s * kH + i], 0.f);
  } else if (p < ow3) {
    const int j = p - ob2;
    for (uint64_t s = 0; s < n; ++s) acc += G2[s * kH + j];
  } else if (p < ob3) {
    const int j = p - ow3;
    for (uint64_t s = 0; s < n; ++s) acc += GO[s] * fmaxf(Z2[s * kH + j], 0.f);
  } else {
    for (uint64_t s = 0; s < n; ++s) acc += GO[s];
  }
  grad[p] = acc;
}

// b1, b2 and their complements ob1 = 1 - b1, ob2 = 1 - b2 come rounded
// from double (1 - 0.999f in float would be 1.3e-5 off 0.001).
__global__ void k_adam(float* __restrict__ th, const float* __restrict__ grad,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float ob1, float ob2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  const float g = grad[p];
  const float mm = b1 * m[p] + ob1 * g;
  const float vv = b2 * v[p] + ob2 * g * g;
  m[p] = mm;
  v[p] = vv;
  th[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void k_to_bf16(const float* __restrict__ th, __nv_bfloat16* __restrict__ tb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) tb[p] = __float2bfloat16_rn(th[p]);
}

// BF16 weights and activations, FP32 accumulation.
__global__ void __launch_bounds__(kH) k_mlp_infer_bf16(const __nv_bfloat16* __restrict__ tb,
                                                       const float* __restrict__ X, uint64_t n,
                                                       float* __restrict__ out) {
  __shared__ __nv_bfloat16 x[kIn], h1[kH];
  __shared__ float red[2];
  const uint64_t s = blockIdx.x;
  const int t = threadIdx.x;
  if (t < kIn) x[t] = __float2bfloat16_rn(X[s * kIn + t]);
  __syncthreads();
  float z1 = __bfloat162float(tb[ob1 + t]);
#pragma unroll
  for (int k = 0; k < kIn; ++k) z1 += __bfloat162float(tb[oW1 + t * kIn + k]) * __bfloat162float(x[k]);
  h1[t] = __float2bfloat16_rn(fmaxf(z1, 0.f));
  __syncthreads();
  float z2 = __bfloat162float(tb[ob2 + t]);
#pragma unroll 16
  for (int i = 0; i < kH; ++i) z2 += __bfloat162float(tb[oW2 + t * kH + i]) * __bfloat162float(h1[i]);
  const float h2 = __bfloat162float(__float2bfloat16_rn(fmaxf(z2, 0.f)));
  const float o = block64_sum(__bfloat162float(tb[ow3 + t]) * h2, red);
  if (t == 0) out[s] = o + __bfloat162float(tb[ob3]);
}

// ---------------------------------------------------------------- features
constexpr int kFT = 1024;
constexpr int kSample = 2048;  // deterministic stride sample per side
constexpr int kSet = 4096;     // open-addressing set of sampled key hashes

__device__ __forceinline__ uint32_t key_hash(const uint32_t* k0, const uint32_t* k1, uint64_t i) {
  const uint32_t h = hash_key(__ldg(k0 + i), k1 ? __ldg(k1 + i) : 0u);
  return h == 0xFFFFFFFFu ? 0xFFFFFFFEu : h;
}

// Inserts h; returns true when it was not yet in the set.
__device__ __forceinline__ bool set_insert(uint32_t* set, uint32_t h) {
  uint32_t s = mix32(h) & (kSet - 1);
  for (int probe = 0; probe < kSet; ++probe) {
    const uint32_t prev = atomicCAS(set + s, 0xFFFFFFFFu, h);
    if (prev == 0xFFFFFFFFu) return true;
    if (prev == h) return false;
    s = (s + 1) & (kSet - 1);
  }
  return false;
}

// Writes the 16 features of one join (see JoinFeatureHost for the host part).
__global__ void __launch_bounds__(kFT) k_join_features(const uint32_t* pk0, const uint32_t* pk1,
                                                       uint64_t np, const uint32_t* bk0,
                                                       const uint32_t* bk1, uint64_t nb,
                                                       JoinFeatureHost hf, float* __restrict__ f) {
  __shared__ uint32_t setP[kSet], setB[kSet];
  __shared__ uint32_t hP[32], hB[32], dB[32], dist[2];
  for (int i = threadIdx.x; i < kSet; i += kFT) setP[i] = setB[i] = 0xFFFFFFFFu;
  if (threadIdx.x < 32) hP[threadIdx.x] = hB[threadIdx.x] = dB[threadIdx.x] = 0;
  if (threadIdx.x < 2) dist[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t sp = np < kSample ? (uint32_t)np : kSample;
  const uint32_t sb = nb < kSample ? (uint32_t)nb : kSample;
  for (uint32_t s = threadIdx.x; s < sp; s += kFT) {
    const uint32_t h = key_hash(pk0, pk1, (uint64_t)s * np / sp);
    atomicAdd(&hP[h >> 27], 1u);
    if (set_insert(setP, h)) atomicAdd(&dist[0], 1u);
  }
  for (uint32_t s = threadIdx.x; s < sb; s += kFT) {
    const uint32_t h = key_hash(bk0, bk1, (uint64_t)s * nb / sb);
    atomicAdd(&hB[h >> 27], 1u);
    if (set_insert(setB, h)) {
      atomicAdd(&dist[1], 1u);
      atomicAdd(&dB[h >> 27], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const float fp = sp ? (float)np / sp : 0.f, fb = sb ? (float)nb / sb : 0.f;
  const float ub_scale = dist[1] ? (float)hf.build_distinct / dist[1] : 0.f;
  float est = 0.f, maxp = 0.f, maxb = 0.f, entp = 0.f, entb = 0.f, dot = 0.f, np2 = 0.f, nb2 = 0.f;
  for (int b = 0; b < 32; ++b) {
    const float cp = hP[b] * fp, cb = hB[b] * fb, db = fmaxf(1.f, dB[b] * ub_scale);
    est += cp * cb / db;
    const float qp = sp ? (float)hP[b] / sp : 0.f, qb = sb ? (float)hB[b] / sb : 0.f;
    maxp = fmaxf(maxp, qp);
    maxb = fmaxf(maxb, qb);
    if (qp > 0.f) entp -= qp * log2f(qp);
    if (qb > 0.f) entb -= qb * log2f(qb);
    dot += qp * qb;
    np2 += qp * qp;
    nb2 += qb * qb;
  }
  f[0] = log2f(1.f + (float)np);
  f[1] = log2f(1.f + (float)nb);
  f[2] = log2f(1.f + hf.probe_full);
  f[3] = log2f(1.f + (float)dist[0]);
  f[4] = log2f(1.f + (float)dist[1]);
  f[5] = log2f(1.f + (float)nb / fmaxf(1.f, hf.build_distinct));
  f[6] = log2f(1.f + est);
  f[7] = maxp;
  f[8] = maxb;
  f[9] = entp;
  f[10] = entb;
  f[11] = (np2 > 0.f && nb2 > 0.f) ? dot * rsqrtf(np2 * nb2) : 0.f;
  f[12] = hf.round;
  f[13] = log2f(1.f + hf.prev_output);
  f[14] = log2f(1.f + hf.prev_delta);
  f[15] = hf.filtered;
}

}  // namespace

cudaError_t mlp_forward(Ctx& c, const float* th, const float* X, uint64_t n, float* out, void* ws) {
  if (n == 0) return cudaSuccess;
  float* Z1 = static_cast<float*>(ws);
  float* Z2 = Z1 + kH * n;
  ProfScope p(c, kMlp, 0.0);
  k_mlp_forward<<<(unsigned)n, kH, 0, c.st>>>(th, X, n, Z1, Z2, out);
  return cudaGetLastError();
}

cudaError_t mlp_gradient(Ctx& c, const float* th, const float* X, const float* y, uint64_t n,
                         float tau, float* out, float* grad, void* ws) {
  if (n == 0) return cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, c.st);
  float* Z1 = static_cast<float*>(ws);
  float* Z2 = Z1 + kH * n;
  float* G1 = Z2 + kH * n;
  float* G2 = G1 + kH * n;
  float* GO = G2 + kH * n;
  ProfScope p(c, kMlp, 0.0);
  k_mlp_forward<<<(unsigned)n, kH, 0, c.st>>>(th, X, n, Z1, Z2, out);
  k_mlp_backward<<<(unsigned)n, kH, 0, c.st>>>(th, y, n, tau, Z1, Z2, out, GO, G1, G2);
  k_mlp_param_grads<<<(kMlpParams + 255) / 256, 256, 0, c.st>>>(X, n, Z1, Z2, GO, G1, G2, grad);
  return cudaGetLastError();
}

cudaError_t mlp_adam(Ctx& c, float* th, const float* grad, float* m, float* v, uint64_t step,
                     float lr) {
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, (double)step));
  const float c2 = (float)(1.0 - std::pow(b2, (double)step));
  ProfScope p(c, kMlp, 0.0);
  k_adam<<<(kMlpParams + 255) / 256, 256, 0, c.st>>>(th, grad, m, v, lr, (float)b1, (float)b2,
                                                      (float)(1.0 - b1), (float)(1.0 - b2), 1e-8f,
                                                      c1, c2);
  return cudaGetLastError();
}

cudaError_t mlp_to_bf16(Ctx& c, const float* th, void* tb) {
  k_to_bf16<<<(kMlpParams + 255) / 256, 256, 0, c.st>>>(th, static_cast<__nv_bfloat16*>(tb));
  return cudaGetLastError();
}

cudaError_t mlp_infer_bf16(Ctx& c, const void* tb, const float* X, uint64_t n, float* out) {
  if (n == 0) return cudaSuccess;
  ProfScope p(c, kMlp, 0.0);
  k_mlp_infer_bf16<<<(unsigned)n, kH, 0, c.st>>>(static_cast<const __nv_bfloat16*>(tb), X, n, out);
  return cudaGetLastError();
}

cudaError_t join_features(Ctx& c, const uint32_t* pk0, const uint32_t* pk1, uint64_t np,
                          const uint32_t* bk0, const uint32_t* bk1, uint64_t nb,
                          const JoinFeatureHost& hf, float* f) {
  ProfScope p(c, kMlp, 4.0 * (np < kSample ? np : kSample) + 4.0 * (nb < kSample ? nb : kSample));
  k_join_features<<<1, kFT, 0, c.st>>>(pk0, pk1, np, bk0, bk1, nb, hf, f);
  return cudaGetLastError();
}

}  // namespace cdl
