// Opt-in per-kernel timing with CUDA events recorded on the launching stream (host side).
#pragma once

#include <cuda_runtime.h>

namespace i4d {

bool profiling_enabled();
// Records a start event now and an end event when the scope closes (no-op when disabled).
class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t st);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  int slot_;
  cudaStream_t st_;
  cudaEvent_t start_;
};

}  // namespace i4d

#define I4D_PROF(name, st) ::i4d::ProfScope i4d_prof_scope_(name, st)
