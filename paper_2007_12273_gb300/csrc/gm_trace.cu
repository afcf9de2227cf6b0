// gm_trace.cu -- per-kernel device times with CUDA events (the library's
// own stage timer).  While a trace is on, the launch code records an event
// on the launching stream after each traced kernel (trace_mark with the
// kernel's name) and one at the start of each API call (a boundary, no
// name).  The time between two consecutive events belongs to the kernel
// named by the later one; a boundary ends an interval without attributing
// it, so host gaps between calls are not counted.  Nothing is recorded
// while the stream is being captured into a CUDA graph.
#include <mutex>
#include <string>
#include <vector>

#include "gm_kernels.cuh"

namespace {

struct Mark {
  cudaEvent_t ev;
  const char* name;  // nullptr: a boundary
};

std::mutex g_tmu;
bool g_on = false;
std::vector<Mark> g_marks;
std::vector<cudaEvent_t> g_pool;
struct Total {
  std::string name;
  double ms;
  int launches;
};
std::vector<Total> g_totals;

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

}  // namespace

void gmcr::trace_mark(const char* name, cudaStream_t s) {
  if (!g_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  cudaEvent_t e = take_event();
  if (!e) return;
  if (cudaEventRecord(e, s) != cudaSuccess) {
    g_pool.push_back(e);
    return;
  }
  g_marks.push_back({e, name});
}

extern "C" {

int gm_trace_begin(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  for (auto& m : g_marks) g_pool.push_back(m.ev);
  g_marks.clear();
  g_totals.clear();
  g_on = true;
  return GM_OK;
}

int gm_trace_end(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_on = false;
  g_totals.clear();
  for (size_t i = 0; i < g_marks.size(); ++i) {
    if (cudaEventSynchronize(g_marks[i].ev) != cudaSuccess)
      return gmcr::record_error(GM_ERR_CUDA, "gm_trace_end: event synchronisation failed");
    if (i == 0 || !g_marks[i].name) continue;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, g_marks[i - 1].ev, g_marks[i].ev) != cudaSuccess) continue;
    size_t k = 0;
    while (k < g_totals.size() && g_totals[k].name != g_marks[i].name) ++k;
    if (k == g_totals.size()) g_totals.push_back({g_marks[i].name, 0.0, 0});
    g_totals[k].ms += ms;
    g_totals[k].launches += 1;
  }
  for (auto& m : g_marks) g_pool.push_back(m.ev);
  g_marks.clear();
  return (int)g_totals.size();
}

int gm_trace_get(int32_t i, char* name, int32_t name_len, double* ms, int32_t* launches) {
  std::lock_guard<std::mutex> lk(g_tmu);
  if (i < 0 || i >= (int)g_totals.size() || !name || name_len < 1 || !ms || !launches)
    return gmcr::record_error(GM_ERR_ARG, "gm_trace_get: index or pointer out of range");
  const std::string& s = g_totals[i].name;
  const size_t n = s.size() < (size_t)(name_len - 1) ? s.size() : (size_t)(name_len - 1);
  s.copy(name, n);
  name[n] = '\0';
  *ms = g_totals[i].ms;
  *launches = g_totals[i].launches;
  return GM_OK;
}

}  // extern "C"
