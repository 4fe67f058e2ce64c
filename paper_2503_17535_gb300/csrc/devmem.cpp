// Stream-ordered device memory pools (devmem.h).
#include "devmem.h"

#include <cstdint>
#include <mutex>

namespace hps {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};
cudaStream_t g_idle_stream[kMaxDevices] = {};

cudaError_t pool_of_current(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t thr = 0;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = pool_of_current(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void dev_free(void* p, cudaStream_t st) {
  if (p && cudaFreeAsync(p, st) != cudaSuccess) cudaGetLastError();
}

void dev_free_idle(void* p) {
  if (!p) return;
  int dev = 0;
  cudaStream_t st = nullptr;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevices) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_idle_stream[dev] && cudaStreamCreateWithFlags(&g_idle_stream[dev], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      g_idle_stream[dev] = nullptr;
    }
    st = g_idle_stream[dev];
  }
  if (cudaFreeAsync(p, st) != cudaSuccess) cudaGetLastError();
}

size_t dev_pool_idle_bytes() {
  cudaMemPool_t pool = nullptr;
  if (pool_of_current(&pool) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  uint64_t reserved = 0, used = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return reserved > used ? (size_t)(reserved - used) : 0;
}

}  // namespace hps
