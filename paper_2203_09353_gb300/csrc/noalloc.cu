// Fixed device scratch for the allocation-free split entry point
// (batched_gemm_fixed_static). The storage is a file-scope __device__ array,
// so it exists as soon as the CUDA runtime loads this file's module on a
// device; nothing here ever calls an allocator.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "bgemm_internal.h"

namespace bg {

namespace {
constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
}  // namespace

size_t static_scratch_capacity() { return kStaticScratchBytes; }

// Resolves the array's address on the current device. The first call on a
// device does the look-up (and so makes the runtime load this module there);
// later calls return the cached address.
bg_status static_scratch(void** out, size_t* bytes, std::string* err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return BG_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *err = "device ordinal beyond the static scratch table";
    return BG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      *err = std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e);
      return BG_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  *bytes = kStaticScratchBytes;
  return BG_OK;
}

}  // namespace bg
