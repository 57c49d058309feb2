// Launch counting and per-kernel-class event timing (diagnostics).
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace qtt {
namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_prof_on{0};

struct Rec {
  int cls;
  cudaEvent_t a, b;
  double flops, bytes;
};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool prof_on() { return g_prof_on.load(std::memory_order_relaxed) != 0; }

ProfToken prof_begin(int cls, cudaStream_t s) {
  ProfToken t{cls, nullptr};
  if (!prof_on()) return t;
  std::lock_guard<std::mutex> lk(g_mu);
  t.ev = get_event();
  if (t.ev) cudaEventRecord(t.ev, s);
  return t;
}

void prof_end(const ProfToken& t, cudaStream_t s, double flops, double bytes) {
  if (!t.ev) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  if (!b) return;
  cudaEventRecord(b, s);
  g_recs.push_back({t.cls, t.ev, b, flops, bytes});
}

}  // namespace qtt

extern "C" {

unsigned long long qtt_kernel_launches(void) { return qtt::g_launches.load(); }

int qtt_profile_enable(int on) {
  qtt::g_prof_on.store(on ? 1 : 0);
  return QTT_OK;
}

int qtt_profile_read(int cls, double* ms, double* flops, double* bytes, long long* launches) {
  std::lock_guard<std::mutex> lk(qtt::g_mu);
  double t = 0, f = 0, b = 0;
  long long n = 0;
  std::vector<qtt::Rec> keep;
  for (auto& r : qtt::g_recs) {
    if (cls >= 0 && r.cls != cls) {
      keep.push_back(r);
      continue;
    }
    float e = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&e, r.a, r.b) == cudaSuccess) {
      t += e;
      f += r.flops;
      b += r.bytes;
      ++n;
    } else {
      cudaGetLastError();
    }
    qtt::g_pool.push_back(r.a);
    qtt::g_pool.push_back(r.b);
  }
  qtt::g_recs.swap(keep);
  if (ms) *ms = t;
  if (flops) *flops = f;
  if (bytes) *bytes = b;
  if (launches) *launches = n;
  return QTT_OK;
}

}  // extern "C"
