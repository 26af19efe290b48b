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

namespace {

// FP32 FMA throughput probe: every thread runs 8 independent packed-FMA chains (16 FMAs per
// iteration per thread), so issue and the FMA pipes, not latency, set the rate.
__global__ void __launch_bounds__(256) fp32_peak_kernel(int iters, float seed, float* __restrict__ out) {
  float2 acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = make_float2(seed + (float)k, seed - (float)k);
  const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = __ffma2_rn(acc[k], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += acc[k].x + acc[k].y;
  if (s == 1234.5f) out[0] = s;  // never true for these inputs; keeps the chains live
}

}  // namespace

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

int32_t i4d_measure_fp32_peak(int32_t blocks_per_sm, int32_t iters, double* tflops, void* stream) {
  if (!tflops || blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1) return I4D_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return I4D_ERR_CUDA;
  float* sink = nullptr;
  if (cudaMallocAsync(&sink, sizeof(float), st) != cudaSuccess) return I4D_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = sms * blocks_per_sm;
  fp32_peak_kernel<<<grid, 256, 0, st>>>(iters / 10 + 1, 1.0f, sink);  // warm-up
  cudaEventRecord(e0, st);
  fp32_peak_kernel<<<grid, 256, 0, st>>>(iters, 1.0f, sink);
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  if (err != cudaSuccess || ms <= 0.0f) return I4D_ERR_CUDA;
  const double flops = (double)grid * 256.0 * (double)iters * 8.0 * 2.0 * 2.0;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return I4D_OK;
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
