// profile.cu -- launch counting and optional CUDA-event timing of every
// library kernel (used by the benchmark to measure kernel durations on the
// stream each kernel runs on).
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dvnr_internal.cuh"

namespace dvnr {

namespace {
struct Record {
  std::string name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
std::vector<Record> g_records;
std::atomic<bool> g_on{false};
std::atomic<int64_t> g_launches{0};
thread_local bool g_capturing = false;
// pinned, device-mapped words into which kernels add the launches of graph
// bodies whose run count only the device knows (conditional WHILE bodies)
std::vector<unsigned long long*> g_dev_counters;
}  // namespace

unsigned long long* device_counter_new() {
  unsigned long long* p = nullptr;
  if (cudaHostAlloc(reinterpret_cast<void**>(&p), sizeof(*p), cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  *p = 0ull;
  std::lock_guard<std::mutex> lk(g_mu);
  g_dev_counters.push_back(p);
  return p;
}

void device_counter_free(unsigned long long* p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < g_dev_counters.size(); ++i)
      if (g_dev_counters[i] == p) {
        g_dev_counters.erase(g_dev_counters.begin() + (std::ptrdiff_t)i);
        break;
      }
    g_launches.fetch_add((int64_t)*reinterpret_cast<volatile unsigned long long*>(p));
  }
  cudaFreeHost(p);
}

bool profiling_on() { return g_on.load(); }
void count_launches(int64_t n) { g_launches.fetch_add(n); }

// How the grouped training ran its steps: graphs captured and replayed, and
// steps launched directly.
std::atomic<int64_t> g_graph_captures{0}, g_graph_replays{0}, g_eager_steps{0};
void count_graph_capture() { g_graph_captures.fetch_add(1); }
void count_graph_replay() { g_graph_replays.fetch_add(1); }
void count_eager_steps(int64_t n) { g_eager_steps.fetch_add(n); }
// launches of each FP16 training kernel enqueued by the host (a launch made
// while a graph is captured counts once, its replays not at all)
std::atomic<int64_t> g_train_plain{0}, g_train_ws{0};
void count_train_launch(bool ws) { (ws ? g_train_ws : g_train_plain).fetch_add(1); }
void set_capturing(bool on) { g_capturing = on; }

ProfScope::ProfScope(const char* name, cudaStream_t s) : name_(name), s_(s) {
  if (g_capturing) return;
  g_launches.fetch_add(1);
  if (!g_on.load()) return;
  if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
    cudaGetLastError();
    a_ = b_ = nullptr;
    return;
  }
  cudaEventRecord(a_, s_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  cudaEventRecord(b_, s_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_records.push_back({name_, a_, b_});
}

}  // namespace dvnr

using namespace dvnr;

extern "C" {

dvnr_status dvnr_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_records) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_records.clear();
  g_on.store(on != 0);
  return DVNR_OK;
}

dvnr_status dvnr_profile_read(const char* kernel, double* total_ms, int64_t* launches) {
  if (!kernel || !total_ms || !launches) {
    set_error("NULL argument");
    return DVNR_E_INVALID;
  }
  DVNR_CUDA(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(g_mu);
  double t = 0.0;
  int64_t n = 0;
  const bool all = std::strcmp(kernel, "*") == 0;
  for (auto& r : g_records) {
    if (!all && r.name != kernel) continue;
    float ms = 0.f;
    DVNR_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    t += ms;
    ++n;
  }
  *total_ms = t;
  *launches = n;
  return DVNR_OK;
}

int64_t dvnr_launch_count(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  int64_t n = g_launches.load();
  for (unsigned long long* p : g_dev_counters) n += (int64_t)*reinterpret_cast<volatile unsigned long long*>(p);
  return n;
}

dvnr_status dvnr_train_kernel_stats(int64_t* plain, int64_t* ws) {
  if (plain) *plain = dvnr::g_train_plain.load();
  if (ws) *ws = dvnr::g_train_ws.load();
  return DVNR_OK;
}

dvnr_status dvnr_graph_stats(int64_t* captures, int64_t* replays, int64_t* eager_steps) {
  if (captures) *captures = dvnr::g_graph_captures.load();
  if (replays) *replays = dvnr::g_graph_replays.load();
  if (eager_steps) *eager_steps = dvnr::g_eager_steps.load();
  return DVNR_OK;
}

}  // extern "C"
