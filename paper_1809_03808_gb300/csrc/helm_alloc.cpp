// Device allocations of the library, counted: every cudaMalloc / cudaFree of
// plan memory goes through dmalloc / dfree, which keep the set of live
// allocations (so a test can see that a failed plan leaks nothing) and can be
// told to fail the k-th next allocation (host-side allocation-failure
// injection; no device fault is involved).
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <unordered_map>

#include "helm.h"
#include "helm_internal.h"

namespace helm {

namespace {

std::mutex g_mu;
std::unordered_map<void*, size_t>& live() {
  static std::unordered_map<void*, size_t> m;
  return m;
}
std::atomic<int> g_fail_countdown{0};  // > 0: the allocation that brings it to 0 fails
std::atomic<int> g_fail_count{0};      // injected failures so far

}  // namespace

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
  const cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return e;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  live()[*ptr] = bytes;
  return cudaSuccess;
}

void dfree(void* ptr) {
  if (!ptr) return;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    live().erase(ptr);
  }
  cudaFree(ptr);
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
    for (const auto& kv : helm::live()) b += kv.second;
    *bytes = b;
  }
  return (int64_t)helm::live().size();
}

}  // extern "C"
