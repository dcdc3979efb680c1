// Opt-in phase tracer: CUDA events recorded on the launching stream around the
// library's internal phases (reduction, sweeps, residuals, fallback, batches),
// summed per phase name when read.  Off by default; leave it off while a
// stream is being captured into a CUDA graph.
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "ssv_internal.cuh"

namespace ssv {

namespace {
struct Span {
  const char* name;
  cudaEvent_t a, b;
};
std::atomic<int> g_on{0};
std::mutex g_mu;
std::vector<Span> g_spans;
}  // namespace

bool trace_on() { return g_on.load(std::memory_order_relaxed) != 0; }

void* trace_begin(const char* name, cudaStream_t st) {
  if (!trace_on()) return nullptr;
  Span* sp = new Span{name, nullptr, nullptr};
  if (cudaEventCreate(&sp->a) != cudaSuccess || cudaEventCreate(&sp->b) != cudaSuccess) {
    delete sp;
    return nullptr;
  }
  cudaEventRecord(sp->a, st);
  return sp;
}

void trace_end(void* tok, cudaStream_t st) {
  if (!tok) return;
  Span* sp = static_cast<Span*>(tok);
  cudaEventRecord(sp->b, st);
  std::lock_guard<std::mutex> lk(g_mu);
  g_spans.push_back(*sp);
  delete sp;
}

}  // namespace ssv

using namespace ssv;

extern "C" {

int ssv_trace_enable(int on) {
  g_on.store(on ? 1 : 0);
  return SSV_OK;
}

int ssv_trace_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& s : g_spans) {
    cudaEventDestroy(s.a);
    cudaEventDestroy(s.b);
  }
  g_spans.clear();
  return SSV_OK;
}

int ssv_trace_read(int max, char* names, int name_len, float* total_ms, int* calls, int* count) {
  if (!count || max < 0 || (max > 0 && (!names || !total_ms || !calls || name_len < 2)))
    return SSV_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<std::string> nm;
  std::vector<float> tot;
  std::vector<int> cnt;
  for (auto& s : g_spans) {
    if (cudaEventSynchronize(s.b) != cudaSuccess) return SSV_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, s.a, s.b);
    size_t k = 0;
    while (k < nm.size() && nm[k] != s.name) ++k;
    if (k == nm.size()) {
      nm.push_back(s.name);
      tot.push_back(0.f);
      cnt.push_back(0);
    }
    tot[k] += ms;
    cnt[k] += 1;
  }
  *count = (int)nm.size();
  for (int k = 0; k < (int)nm.size() && k < max; ++k) {
    std::string t = nm[k].substr(0, (size_t)name_len - 1);
    for (size_t c = 0; c < t.size(); ++c) names[(size_t)k * name_len + c] = t[c];
    names[(size_t)k * name_len + t.size()] = '\0';
    total_ms[k] = tot[k];
    calls[k] = cnt[k];
  }
  return SSV_OK;
}

}  // extern "C"
