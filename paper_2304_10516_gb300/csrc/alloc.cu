// alloc.cu -- every device allocation of libdvnr goes through these wrappers,
// which keep a table of the allocations the library holds (address -> bytes)
// and can be told to fail the n-th allocation from now, as if the device were
// out of memory, so that tests drive each call's cleanup path on the host and
// check that nothing leaks (dvnr_debug_fail_alloc, dvnr_debug_live_allocs).
#include <atomic>
#include <mutex>
#include <unordered_map>

#include "dvnr_internal.cuh"

namespace dvnr {

namespace {
std::mutex g_alloc_mu;
std::unordered_map<void*, size_t> g_live;
std::atomic<int64_t> g_fail_countdown{0};

// True for the allocation that the armed countdown reaches (then disarmed).
bool injected_failure() {
  int64_t c = g_fail_countdown.load();
  while (c > 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
  }
  return false;
}

void remember(void* p, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_live[p] = bytes;
}

void forget(void* p) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_live.erase(p);
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) remember(*p, bytes);
  return e;
}

cudaError_t dev_free(void* p) {
  if (!p) return cudaSuccess;
  forget(p);
  return cudaFree(p);
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e == cudaSuccess) remember(*p, bytes);
  return e;
}

cudaError_t dev_free_async(void* p, cudaStream_t s) {
  if (!p) return cudaSuccess;
  forget(p);
  return cudaFreeAsync(p, s);
}

}  // namespace dvnr

extern "C" dvnr_status dvnr_debug_fail_alloc(int64_t nth) {
  if (nth < 0) {
    dvnr::set_error("nth must be >= 0");
    return DVNR_E_INVALID;
  }
  dvnr::g_fail_countdown.store(nth);
  return DVNR_OK;
}

extern "C" dvnr_status dvnr_debug_live_allocs(int64_t* count, int64_t* bytes) {
  std::lock_guard<std::mutex> lk(dvnr::g_alloc_mu);
  int64_t b = 0;
  for (const auto& kv : dvnr::g_live) b += (int64_t)kv.second;
  if (count) *count = (int64_t)dvnr::g_live.size();
  if (bytes) *bytes = b;
  return DVNR_OK;
}
