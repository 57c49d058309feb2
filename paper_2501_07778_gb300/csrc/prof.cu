// Launch counting and per-kernel-class event timing (diagnostics).
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace qtt {
namespace {
std::atomic<unsigned long long> g_launches{0};
std::atomic<unsigned long long> g_allocs{0};
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
void count_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

int num_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 1;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();
    return 1;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

namespace {
// Eight independent FMA chains per thread: the rate of the FMA pipe of the
// given precision when every SM holds enough warps.  The chains' sum is
// stored so that nothing is optimised away.
template <typename T>
__global__ void __launch_bounds__(256) fma_chain_kernel(int iters, T a, T b, T* sink) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  T acc = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) acc += x[c];
  sink[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = acc;
}
}  // namespace

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

unsigned long long qtt_device_allocations(void) { return qtt::g_allocs.load(); }

int qtt_measure_fma_peak(int prec, double* tflops, void* stream) {
  try {
    QTT_REQUIRE(tflops && (prec == QTT_F64 || prec == QTT_F32), "qtt_measure_fma_peak: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int blocks = qtt::num_sms() * 8, threads = 256;
    // about 20 ms of work at the nominal rate of each precision
    const int iters = prec == QTT_F64 ? 4096 : 262144;
    struct Res {   // released on every path
      void* sink = nullptr;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      ~Res() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (sink) cudaFree(sink);
      }
    } r;
    qtt::count_alloc();
    QTT_CUDA(cudaMalloc(&r.sink, (size_t)blocks * threads * 8));
    QTT_CUDA(cudaEventCreate(&r.e0));
    QTT_CUDA(cudaEventCreate(&r.e1));
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // the first launch warms up clocks and caches
      QTT_CUDA(cudaEventRecord(r.e0, s));
      if (prec == QTT_F64)
        qtt::fma_chain_kernel<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, (double*)r.sink);
      else
        qtt::fma_chain_kernel<float><<<blocks, threads, 0, s>>>(iters, 0.9999f, 1e-4f, (float*)r.sink);
      QTT_CHECK_LAUNCH();
      QTT_CUDA(cudaEventRecord(r.e1, s));
      QTT_CUDA(cudaEventSynchronize(r.e1));
      QTT_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
    }
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    *tflops = ms > 0 ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return QTT_OK;
  } catch (const qtt::QttError& e) {
    qtt::set_last_error(e.what());
    return e.code;
  }
}

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
