// Dense relations as bitmaps, a second form of step (c) of the round
// (Section 4, "Projection and Selection" and the sort + unique that
// follows).  Where a relation's tuples fit in 2^T bits, new tuples set bits
// instead of being written, sorted and deduplicated.  Extraction reads the
// bits back in increasing order: the same sorted unique list the radix sort
// and the unique pass produce, at the cost of one pass over the bitmap.
#include "kernels.h"

namespace cdl {

namespace {

constexpr int kXT = 256;                              // threads per extraction block
constexpr int kXWords = 8;                            // bitmap words per thread
constexpr uint64_t kXTile = (uint64_t)kXT * kXWords;  // words per block

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

__host__ __device__ __forceinline__ uint64_t words_of(uint64_t nbits) {
  return nbits >= 32 ? nbits >> 5 : 1;
}

__global__ void __launch_bounds__(256) k_dense_insert(DenseSet d, ColsIn rows, uint64_t n,
                                                      uint32_t* err) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x; b < n; b += stride) {
    const uint64_t i = b + threadIdx.x;
    const bool keep = i < n;
    uint32_t v[kMaxK] = {0, 0, 0, 0};
    if (keep) {
#pragma unroll
      for (int k = 0; k < kMaxK; ++k)
        if (k < (int)d.k) v[k] = __ldg(rows.c[k] + i);
    }
    dense_set_bits(d, v, keep, err);
  }
}

// The words a thread owns: [w0, w0 + kXWords) clipped to nw.
__device__ __forceinline__ void load_words(const uint32_t* words, uint64_t w0, uint64_t nw,
                                           uint32_t (&w)[kXWords]) {
  if (w0 + kXWords <= nw) {  // 32-byte aligned: w0 is a multiple of 8
    const uint4 a = *reinterpret_cast<const uint4*>(words + w0);
    const uint4 b = *reinterpret_cast<const uint4*>(words + w0 + 4);
    w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w;
    w[4] = b.x, w[5] = b.y, w[6] = b.z, w[7] = b.w;
  } else {
#pragma unroll
    for (int i = 0; i < kXWords; ++i) w[i] = w0 + i < nw ? words[w0 + i] : 0u;
  }
}

__global__ void __launch_bounds__(kXT) k_dense_count(const uint32_t* __restrict__ words,
                                                     uint64_t nw, uint32_t* __restrict__ counts) {
  __shared__ uint32_t red[kXT / 32 + 1];
  const uint64_t w0 = (uint64_t)blockIdx.x * kXTile + (uint64_t)threadIdx.x * kXWords;
  uint32_t w[kXWords];
  load_words(words, w0, nw, w);
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < kXWords; ++i) c += __popc(w[i]);
  uint32_t total;
  block_exclusive_sum<kXT, uint32_t>(c, red, &total);
  if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// Rows of the set bits at their ranks, in bit order; the words are cleared
// behind the read so that the bitmap starts the next round empty.
__global__ void __launch_bounds__(kXT) k_dense_write(DenseSet d, uint64_t nw,
                                                     const uint64_t* __restrict__ offs,
                                                     ColsOut out, uint64_t cap, uint32_t* err) {
  __shared__ uint32_t red[kXT / 32 + 1];
  const uint64_t w0 = (uint64_t)blockIdx.x * kXTile + (uint64_t)threadIdx.x * kXWords;
  uint32_t w[kXWords];
  load_words(d.words, w0, nw, w);
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < kXWords; ++i) c += __popc(w[i]);
  uint32_t total;
  uint64_t pos = offs[blockIdx.x] + block_exclusive_sum<kXT, uint32_t>(c, red, &total);
#pragma unroll
  for (int i = 0; i < kXWords; ++i) {
    uint32_t x = w[i];
    if (x) d.words[w0 + i] = 0u;
    while (x) {
      const uint64_t idx = ((w0 + i) << 5) | (uint64_t)(__ffs(x) - 1);
      x &= x - 1;
      if (pos < cap) {
#pragma unroll
        for (int k = 0; k < kMaxK; ++k)
          if (k < (int)d.k) out.c[k][pos] = (uint32_t)(idx >> d.shift[k]) & d.mask[k];
      } else {
        atomicOr(err, kErrCapacity);
      }
      ++pos;
    }
  }
}

}  // namespace

cudaError_t dense_insert(Ctx& c, const DenseSet& d, ColsIn rows, uint64_t n) {
  if (n == 0) return cudaSuccess;
  ProfScope p(c, kDense, 4.0 * d.k * n);
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_dense_insert<<<(unsigned)blocks, 256, 0, c.st>>>(d, rows, n, c.d_err);
  return cudaGetLastError();
}

size_t dense_extract_workspace(uint64_t nbits) {
  const uint64_t tiles = (words_of(nbits) + kXTile - 1) / kXTile;
  return up256(tiles * 4) + up256(tiles * 8) + scan_workspace(tiles);
}

cudaError_t dense_extract(Ctx& c, const DenseSet& d, ColsOut out, uint64_t cap,
                          uint64_t* d_count, void* ws) {
  const uint64_t nw = words_of(d.nbits);
  const uint64_t tiles = (nw + kXTile - 1) / kXTile;
  char* w = static_cast<char*>(ws);
  uint32_t* counts = reinterpret_cast<uint32_t*>(w);
  w += up256(tiles * 4);
  uint64_t* offs = reinterpret_cast<uint64_t*>(w);
  w += up256(tiles * 8);
  {
    ProfScope p(c, kDense, 4.0 * nw);
    k_dense_count<<<(unsigned)tiles, kXT, 0, c.st>>>(d.words, nw, counts);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = exclusive_scan(c, counts, tiles, offs, d_count, w);
  if (e != cudaSuccess) return e;
  // the bitmap read again and its set words cleared; the rows are added
  // to the class's bytes once their number is known
  ProfScope p(c, kDense, 4.0 * nw);
  k_dense_write<<<(unsigned)tiles, kXT, 0, c.st>>>(d, nw, offs, out, cap, c.d_err);
  return cudaGetLastError();
}

}  // namespace cdl
