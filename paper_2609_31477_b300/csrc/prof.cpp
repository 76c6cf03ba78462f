// Launch counter and per-kernel-kind CUDA-event timing (opt-in per case).
#include <atomic>

#include "viv_internal.h"

namespace viv {

static std::atomic<int64_t> g_launches{0};
thread_local Profiler* g_prof = nullptr;

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches() { return g_launches.load(); }

void Profiler::start(int k, cudaStream_t s) {
  if (used + 2 > ev.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      VIV_CUDA(cudaEventCreate(&e));
      ev.push_back(e);
    }
    kind.resize(ev.size() / 2 + 1);
    level.resize(ev.size() / 2 + 1);
  }
  kind[used / 2] = k;
  level[used / 2] = cur_level;
  VIV_CUDA(cudaEventRecord(ev[used], s));
  ++used;
}

void Profiler::stop(cudaStream_t s) {
  VIV_CUDA(cudaEventRecord(ev[used], s));
  ++used;
}

void Profiler::read(double* ms, int64_t* count) {
  for (int k = 0; k < K_NKINDS; ++k) {
    ms[k] = 0;
    count[k] = 0;
  }
  if (used) VIV_CUDA(cudaEventSynchronize(ev[used - 1]));
  level_ms.clear();
  for (size_t i = 0; i + 1 < used; i += 2) {
    float t = 0;
    VIV_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
    ms[kind[i / 2]] += t;
    count[kind[i / 2]] += 1;
    const int l = level[i / 2];
    if (l >= 0) {
      if ((int)level_ms.size() < (l + 1) * K_NKINDS) level_ms.resize((l + 1) * K_NKINDS, 0.0);
      level_ms[l * K_NKINDS + kind[i / 2]] += t;
    }
  }
  used = 0;
}

void prof_level(int l) {
  if (g_prof) g_prof->cur_level = l;
}

Profiler::~Profiler() {
  for (auto e : ev) cudaEventDestroy(e);
}

}  // namespace viv
