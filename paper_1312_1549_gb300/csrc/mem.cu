// Device memory of the library's contexts: stream-ordered allocations from a memory pool the
// library owns, one per device. A freed block stays in the pool for the next context instead of
// going back to the driver: cudaFree waits for the whole device and unmaps the pages, and a
// context of the Si512 workload holds about forty buffers (several GB), so creating and
// releasing contexts one after another (benchmarks, batches, warm-started sequences that
// rebuild their setup) would otherwise pay for that every time.
#include "omm_internal.cuh"

#include <cstdint>
#include <map>
#include <mutex>
#include <new>

namespace omm {
namespace mem {
namespace {

std::mutex g_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t pool_of_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    throw std::bad_alloc();
  }
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    throw std::bad_alloc();
  }
  uint64_t keep = UINT64_MAX;  // keep freed memory for reuse (no release at synchronisation points)
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  g_pools[dev] = pool;
  return pool;
}

}  // namespace

void* alloc(size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = pool_of_current_device();
  void* p = nullptr;
  if (cudaMallocFromPoolAsync(&p, bytes ? bytes : 1, pool, st) != cudaSuccess) {
    cudaGetLastError();
    throw std::bad_alloc();
  }
  return p;
}

void release(void* p, cudaStream_t st) {
  if (p == nullptr) return;
  if (cudaFreeAsync(p, st) != cudaSuccess) cudaGetLastError();
}

}  // namespace mem
}  // namespace omm
