// Device memory of the contexts: stream-ordered allocations from one memory pool per device.
//
// Creating a context allocates a few dozen buffers (1-8 GB at 1024^2 cells, S16) and destroying it frees them;
// through cudaMalloc / cudaFree every context maps and unmaps that memory again.  The pool keeps up to kKeepBytes
// reserved after frees (its release threshold), so the next context of a similar size reuses the mapping.  Every
// allocation is ordered on the legacy default stream and synchronised before it is handed out, so any stream may
// use it; every free waits for the device first, since the buffer may still be read by kernels on another stream.
// If the pool cannot be created on a device, allocations there fall back to cudaMalloc / cudaFree.
#include <cstdint>
#include <mutex>

#include "lmdg_internal.h"

namespace lmdg {
namespace {

constexpr int kMaxDevices = 64;
constexpr uint64_t kKeepBytes = uint64_t(16) << 30;   // memory the pool keeps reserved after frees

struct DevicePool {
  bool tried = false;
  cudaMemPool_t pool = nullptr;
};
DevicePool g_pools[kMaxDevices];
std::mutex g_mu;

cudaMemPool_t pool_of_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  DevicePool &d = g_pools[dev];
  if (!d.tried) {
    d.tried = true;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) == cudaSuccess) {
      uint64_t keep = kKeepBytes;
      if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess) {
        d.pool = p;
      } else {
        cudaMemPoolDestroy(p);
      }
    }
    cudaGetLastError();   // a refused pool leaves no error behind: the fallback runs
  }
  return d.pool;
}

}  // namespace

cudaError_t dalloc(void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  cudaMemPool_t pool = pool_of_current_device();
  if (!pool) return cudaMalloc(p, bytes);
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, cudaStreamLegacy);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  e = cudaStreamSynchronize(cudaStreamLegacy);
  if (e != cudaSuccess) {
    cudaFreeAsync(*p, cudaStreamLegacy);
    *p = nullptr;
  }
  return e;
}

void dfree(void *p) {
  if (!p) return;
  if (!pool_of_current_device()) {
    cudaFree(p);
    return;
  }
  cudaDeviceSynchronize();
  cudaFreeAsync(p, cudaStreamLegacy);
}

}  // namespace lmdg
