// Launch statistics per kernel class (cbc_stats_* of cbc.h).
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "planner.h"

namespace cbc {
namespace {
struct Pending {
  int cls;
  cudaEvent_t a, b;
};
std::mutex g_mu;
cbc_stats g_stats{};
bool g_timing = false;
std::vector<Pending> g_pending;
}  // namespace

void note_launches(int cls, int n) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_stats.launches[cls] += n;
}

void note_flops(int cls, double flops) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_stats.flops[cls] += flops;
}

KTimer::KTimer(int cls_, cudaStream_t s_, int64_t launches, double flops) : cls(cls_), s(s_) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_stats.launches[cls] += launches;
  g_stats.flops[cls] += flops;
  g_stats.groups[cls] += 1;
  if (g_timing) {
    cudaEventCreate(&e0);
    cudaEventRecord(e0, s);
  }
}

KTimer::~KTimer() {
  if (!e0) return;
  cudaEvent_t e1;
  cudaEventCreate(&e1);
  cudaEventRecord(e1, s);
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back({cls, e0, e1});
}

}  // namespace cbc

using namespace cbc;

extern "C" {

int cbc_stats_enable(int timing) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_timing = timing != 0;
  return CBC_OK;
}

int cbc_stats_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    cudaEventSynchronize(p.b);
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_pending.clear();
  g_stats = cbc_stats{};
  return CBC_OK;
}

int cbc_stats_read(cbc_stats* out) {
  if (!out) return fail(CBC_ERR_INVALID_ARG, "cbc_stats_read: NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& p : g_pending) {
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e != cudaSuccess) return cuda_fail(e, "cbc_stats_read");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    g_stats.ms[p.cls] += ms;
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_pending.clear();
  *out = g_stats;
  return CBC_OK;
}

}  // extern "C"
