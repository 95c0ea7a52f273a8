// Launch counting and CUDA-event timing of the march's decoder-MLP launches.
#include <vector>

#include "common.cuh"

namespace dist {

namespace {
constexpr int kMaxTimed = 65536;
struct Prof {
  bool on = false;
  long long launches = 0;
  std::vector<cudaEvent_t> ev;   // (start, end) pairs
  std::vector<int> kind;         // kernel kind of each pair
  int used = 0;                  // events in use
  int open_kind = -1;
};
Prof g_prof;
}  // namespace

void count_launch(int n) {
  if (g_prof.on) g_prof.launches += n;
}

void prof_mlp_begin(cudaStream_t st, int kind) {
  g_prof.open_kind = -1;
  if (!g_prof.on || g_prof.used / 2 >= kMaxTimed) return;
  if (g_prof.used + 2 > (int)g_prof.ev.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      g_prof.ev.push_back(e);
    }
  }
  if (cudaEventRecord(g_prof.ev[g_prof.used], st) == cudaSuccess) g_prof.open_kind = kind;
}

void prof_mlp_end(cudaStream_t st) {
  if (!g_prof.on || g_prof.open_kind < 0) return;
  if (cudaEventRecord(g_prof.ev[g_prof.used + 1], st) != cudaSuccess) return;
  if ((int)g_prof.kind.size() < g_prof.used / 2 + 1) g_prof.kind.resize(g_prof.used / 2 + 1);
  g_prof.kind[g_prof.used / 2] = g_prof.open_kind;
  g_prof.used += 2;
  g_prof.open_kind = -1;
}

}  // namespace dist

using namespace dist;

extern "C" {

dist_status dist_profile_enable(int enable) {
  g_prof.on = enable != 0;
  if (enable) {
    g_prof.launches = 0;
    g_prof.used = 0;
  }
  return DIST_OK;
}

dist_status dist_profile_read(double* mlp_ms, int64_t* mlp_launches, int64_t* all_launches) {
  double ms[3] = {0.0, 0.0, 0.0};
  int64_t cnt[3] = {0, 0, 0};
  for (int i = 0; i + 1 < g_prof.used; i += 2) {
    DIST_CUDA_TRY(cudaEventSynchronize(g_prof.ev[i + 1]));
    float t = 0.f;
    DIST_CUDA_TRY(cudaEventElapsedTime(&t, g_prof.ev[i], g_prof.ev[i + 1]));
    const int k = g_prof.kind[i / 2];
    ms[k] += t;
    cnt[k] += 1;
  }
  for (int k = 0; k < 3; ++k) {
    if (mlp_ms) mlp_ms[k] = ms[k];
    if (mlp_launches) mlp_launches[k] = cnt[k];
  }
  if (all_launches) *all_launches = g_prof.launches;
  return DIST_OK;
}

}  // extern "C"
