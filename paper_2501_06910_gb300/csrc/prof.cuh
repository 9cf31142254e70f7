// prof.cuh -- optional per-kernel device timing with CUDA events (off by
// default). Each launch site wraps its launch in PROF_SCOPE(name, stream):
// when profiling is on, events recorded on the launch stream bracket the
// kernel and mcc_profile_read accumulates their elapsed times by name.
#pragma once
#include <cuda_runtime.h>

namespace mcc {
extern bool g_profile_on;
void prof_record(const char *name, cudaStream_t s, bool begin);

struct ProfScope {
  const char *name;
  cudaStream_t s;
  ProfScope(const char *n, cudaStream_t st) : name(n), s(st) {
    if (g_profile_on) prof_record(name, s, true);
  }
  ~ProfScope() {
    if (g_profile_on) prof_record(name, s, false);
  }
};
}  // namespace mcc

#define MCC_CAT2(a, b) a##b
#define MCC_CAT(a, b) MCC_CAT2(a, b)
#define PROF_SCOPE(name, stream) mcc::ProfScope MCC_CAT(prof_scope_, __LINE__)(name, stream)
