// Device allocations of the library, counted: every allocation and free of
// plan memory goes through dmalloc / dfree, which keep the set of live
// allocations (so a test can see that a failed plan leaks nothing) and can be
// told to fail the k-th next allocation (host-side allocation-failure
// injection; no device fault is involved).
//
// Allocations are stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// legacy stream) rather than cudaMalloc / cudaFree: cudaFree waits for the
// whole device, so building or destroying a plan would stall every stream's
// work in flight (a request server's other requests).  An allocation is
// ordered before any later work by a wait on the legacy stream alone; a free
// is issued only after the plan's own streams have finished with it.
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <unordered_map>

#include "helm.h"
#include "helm_internal.h"

namespace helm {

namespace {

struct Alloc {
  size_t bytes;
  bool pool;  // from the stream-ordered allocator (else plain cudaMalloc)
};
std::mutex g_mu;
std::unordered_map<void*, Alloc>& live() {
  static std::unordered_map<void*, Alloc> m;
  return m;
}
std::atomic<int> g_fail_countdown{0};  // > 0: the allocation that brings it to 0 fails
std::atomic<int> g_fail_count{0};      // injected failures so far

}  // namespace

cudaError_t allow_dynamic_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;  // (kernel, device) -> bytes allowed
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[{func, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

cudaError_t dmalloc(void** ptr, size_t bytes) {
  *ptr = nullptr;
  int c = g_fail_countdown.load();
  while (c > 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) {
      if (c == 1) {
        g_fail_count.fetch_add(1);
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  bool pool = true;
  cudaError_t e = cudaMallocAsync(ptr, bytes, nullptr);
  if (e == cudaErrorNotSupported) {  // no memory pools on this device: plain allocation
    cudaGetLastError();
    pool = false;
    e = cudaMalloc(ptr, bytes);
  } else if (e == cudaSuccess) {
    e = cudaStreamSynchronize(nullptr);
  }
  if (e != cudaSuccess) {
    if (*ptr) pool ? cudaFreeAsync(*ptr, nullptr) : cudaFree(*ptr);
    *ptr = nullptr;
    cudaGetLastError();
    return e;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  live()[*ptr] = Alloc{bytes, pool};
  return cudaSuccess;
}

void dfree(void* ptr) {
  if (!ptr) return;
  bool pool = true;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = live().find(ptr);
    if (it != live().end()) {
      pool = it->second.pool;
      live().erase(it);
    }
  }
  if (pool) cudaFreeAsync(ptr, nullptr);
  else cudaFree(ptr);
}

}  // namespace helm

extern "C" {

int helm_debug_fail_alloc(int k) {
  helm::g_fail_countdown.store(k > 0 ? k : 0);
  return helm::g_fail_count.load();
}

int64_t helm_debug_live_allocations(size_t* bytes) {
  std::lock_guard<std::mutex> lk(helm::g_mu);
  if (bytes) {
    size_t b = 0;
    for (const auto& kv : helm::live()) b += kv.second.bytes;
    *bytes = b;
  }
  return (int64_t)helm::live().size();
}

}  // extern "C"
