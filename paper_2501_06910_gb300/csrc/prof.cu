// prof.cu -- per-kernel event timing behind mcc_profile_* (diagnostics).
#include <cuda_runtime.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mcc.h"
#include "prof.cuh"

namespace mcc {
bool g_profile_on = false;

namespace {
struct Pending {
  std::string name;
  cudaEvent_t a, b;
};
struct Acc {
  double ms = 0.0;
  long long n = 0;
};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;
std::map<std::string, Acc> g_acc;
std::map<std::string, size_t> g_open;  // name -> index in g_pending of an open pair

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void drain() {
  for (auto &p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      Acc &a = g_acc[p.name];
      a.ms += ms;
      a.n += 1;
    }
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
  g_open.clear();
}
}  // namespace

void prof_record(const char *name, cudaStream_t s, bool begin) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (begin) {
    Pending p{name, take_event(), take_event()};
    cudaEventRecord(p.a, s);
    g_open[name] = g_pending.size();
    g_pending.push_back(p);
  } else {
    auto it = g_open.find(name);
    if (it == g_open.end()) return;
    cudaEventRecord(g_pending[it->second].b, s);
    g_open.erase(it);
  }
}
}  // namespace mcc

extern "C" void mcc_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(mcc::g_mu);
  mcc::g_profile_on = on != 0;
}

extern "C" void mcc_profile_reset(void) {
  std::lock_guard<std::mutex> lk(mcc::g_mu);
  mcc::drain();
  mcc::g_acc.clear();
}

extern "C" int mcc_profile_read(char (*names)[32], double *ms, long long *launches, int max_entries) {
  std::lock_guard<std::mutex> lk(mcc::g_mu);
  mcc::drain();
  int i = 0;
  for (auto &kv : mcc::g_acc) {
    if (i >= max_entries) break;
    strncpy(names[i], kv.first.c_str(), 31);
    names[i][31] = 0;
    ms[i] = kv.second.ms;
    launches[i] = kv.second.n;
    i++;
  }
  return i;
}
