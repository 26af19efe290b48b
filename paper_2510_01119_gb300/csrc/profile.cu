// Opt-in kernel timing: a start/end CUDA event pair per launch, summed per kernel name on read.
#include <mutex>
#include <string.h>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "profile.cuh"

namespace i4d {

namespace {

struct Entry {
  std::string name;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  double total_ms = 0.0;
  long long launches = 0;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Entry> g_entries;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int slot_for(const char* name) {
  for (size_t k = 0; k < g_entries.size(); ++k)
    if (g_entries[k].name == name) return (int)k;
  g_entries.push_back(Entry{name, {}, 0.0, 0});
  return (int)g_entries.size() - 1;
}

void drain(Entry& e) {
  for (auto& pr : e.pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(pr.second) == cudaSuccess && cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
      e.total_ms += ms;
      e.launches += 1;
    }
    g_pool.push_back(pr.first);
    g_pool.push_back(pr.second);
  }
  e.pending.clear();
}

}  // namespace

bool profiling_enabled() { return g_on; }

ProfScope::ProfScope(const char* name, cudaStream_t st) : slot_(-1), st_(st), start_(nullptr) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  start_ = take_event();
  if (!start_) return;
  if (cudaEventRecord(start_, st_) != cudaSuccess) {
    g_pool.push_back(start_);
    start_ = nullptr;
    return;
  }
  slot_ = slot_for(name);
}

ProfScope::~ProfScope() {
  if (slot_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t end = take_event();
  if (!end || cudaEventRecord(end, st_) != cudaSuccess) {
    g_pool.push_back(start_);
    if (end) g_pool.push_back(end);
    return;
  }
  g_entries[slot_].pending.emplace_back(start_, end);
}

}  // namespace i4d

using namespace i4d;

extern "C" {

int32_t i4d_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return I4D_OK;
}

void i4d_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& e : g_entries) {
    drain(e);
    e.total_ms = 0.0;
    e.launches = 0;
  }
}

int32_t i4d_profile_count(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  return (int32_t)g_entries.size();
}

int32_t i4d_profile_read(int32_t k, char* name, int32_t name_len, double* total_ms, int64_t* launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (k < 0 || k >= (int32_t)g_entries.size() || !total_ms || !launches) return I4D_ERR_ARG;
  Entry& e = g_entries[k];
  drain(e);
  if (name && name_len > 0) {
    strncpy(name, e.name.c_str(), (size_t)name_len - 1);
    name[name_len - 1] = '\0';
  }
  *total_ms = e.total_ms;
  *launches = e.launches;
  return I4D_OK;
}

}  // extern "C"
