// The static device scratch of top_propagate_noalloc, in a translation unit of its own: its
// module (and so the array) is loaded on a device only when this unit's symbol is first used
// there (the first no-alloc call), or for every context when CUDA loads modules eagerly
// (CUDA_MODULE_LOADING=EAGER). Processes that only use handle calls never pay for it under the
// default lazy loading.
#include <mutex>

#include "top_aux.h"

namespace top {

static __device__ __align__(256) unsigned char g_noalloc_scratch[TOP_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoallocDevices = 64;
std::mutex g_mutex;
void* g_addr[kNoallocDevices] = {};
}  // namespace

cudaError_t noalloc_scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoallocDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace top
