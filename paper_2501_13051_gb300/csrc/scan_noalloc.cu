// Exclusive scan for callers that cannot allocate device memory.
//
// cdl_exclusive_scan needs a caller-provided workspace for its per-tile
// sums.  Some callers cannot provide one: code running where cudaMalloc is
// not allowed or not wanted (inside a larger framework's allocation-free
// region, a plugin given only the input and output pointers, a hot path that
// must never touch the allocator).  This variant keeps that scratch in a
// fixed array in the library's own device memory instead, so it allocates
// nothing.  The array is a file-scope __device__ variable: every GPU on
// which the library's module is loaded holds it until the process exits.
#include <mutex>

#include "kernels.h"

namespace {

// Scratch: 65,536 tile sums plus the total, 512 KiB + 8 bytes per GPU.
constexpr uint64_t kNoAllocTiles = 1ull << 16;
constexpr uint64_t kNoAllocMaxN = kNoAllocTiles * cdl::kScanTile;  // 134,217,728 counts

static __device__ __align__(256) uint64_t g_scan_scratch[kNoAllocTiles + 1];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint64_t* g_scratch_addr[kMaxDevices] = {};  // device address of g_scan_scratch per GPU

}  // namespace

extern "C" cdl_status cdl_exclusive_scan_noalloc(const uint32_t* in, uint64_t n, uint64_t* out,
                                                 uint64_t* total_host, void* stream) {
  if ((!in || !out) && n) return CDL_E_INVALID;
  if (n > kNoAllocMaxN) return CDL_E_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CDL_E_CUDA;
  uint64_t* scratch = nullptr;
  {
    // In host code g_scan_scratch names a host-side stand-in, not device
    // memory: the device address comes from the runtime, once per GPU, with
    // that GPU current.
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scan_scratch) != cudaSuccess || !p) return CDL_E_CUDA;
      g_scratch_addr[dev] = static_cast<uint64_t*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cdl::Ctx c;
  c.st = st;
  uint64_t* d_total = scratch + kNoAllocTiles;
  // Every tile sum and the total are written by this call before they are
  // read, so nothing left by an earlier call leaks into the result.
  if (cdl::exclusive_scan(c, in, n, out, d_total, scratch) != cudaSuccess) return CDL_E_CUDA;
  if (total_host) {
    cudaError_t e = cudaMemcpyAsync(total_host, d_total, sizeof(uint64_t),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return CDL_E_CUDA;
  }
  return CDL_OK;
}
