// prof.cu -- per-kernel event timing behind mcc_profile_* (diagnostics).
// Every bracketed launch registers one (begin, end) event pair that stays
// registered until mcc_profile_reset. A read sums, per kernel name, the
// elapsed time of each pair's latest recording: for eager launches every
// launch owns a pair; when the launches were captured into a CUDA graph, each
// replay re-records the captured pairs and a read after a replay returns that
// replay's times.
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
struct Pair {
  std::string name;
  cudaEvent_t a, b;
  bool closed;
};
std::mutex g_mu;
std::vector<Pair> g_pairs;
std::map<std::string, size_t> g_open;  // name -> index of an open pair
}  // namespace

// Inside stream capture an event record becomes a timing node of the graph
// only with cudaEventRecordExternal.
static void record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}

void prof_record(const char *name, cudaStream_t s, bool begin) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (begin) {
    Pair p{name, nullptr, nullptr, false};
    if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) return;
    record(p.a, s);
    g_open[name] = g_pairs.size();
    g_pairs.push_back(p);
  } else {
    auto it = g_open.find(name);
    if (it == g_open.end()) return;
    record(g_pairs[it->second].b, s);
    g_pairs[it->second].closed = true;
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
  for (auto &p : mcc::g_pairs) {
    cudaEventSynchronize(p.b);
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  mcc::g_pairs.clear();
  mcc::g_open.clear();
}

extern "C" int mcc_profile_read(char (*names)[32], double *ms, long long *launches, int max_entries) {
  std::lock_guard<std::mutex> lk(mcc::g_mu);
  std::map<std::string, std::pair<double, long long>> acc;
  for (auto &p : mcc::g_pairs) {
    if (!p.closed) continue;
    float t = 0.f;
    if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&t, p.a, p.b) != cudaSuccess)
      continue;
    auto &e = acc[p.name];
    e.first += t;
    e.second += 1;
  }
  int i = 0;
  for (auto &kv : acc) {
    if (i >= max_entries) break;
    strncpy(names[i], kv.first.c_str(), 31);
    names[i][31] = 0;
    ms[i] = kv.second.first;
    launches[i] = kv.second.second;
    i++;
  }
  return i;
}
