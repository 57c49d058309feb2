// qtt_solve_batched: many independent solves (uneven levels, patch counts
// and ranks) drained from one work queue by worker threads, each issuing its
// solve's kernels on its own non-blocking stream.  One AMEn step is a chain
// of small dependent contractions that cannot fill the SMs, so concurrent
// solves are what keeps the GPU busy; the caller's stream waits on every
// worker stream before the call returns its results.
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace qtt {
int solve(const qtt_tensor* K, const qtt_tensor* f, const qtt_tensor* x0, const qtt_tensor* z0,
          const qtt_solve_opts* opts, qtt_tensor** xout, qtt_solve_info* info, cudaStream_t s);
void set_gpu_share(int n);
}

using namespace qtt;

extern "C" int qtt_solve_batched(int count, const qtt_tensor* const* K, const qtt_tensor* const* f,
                                 const qtt_tensor* const* x0, const qtt_solve_opts* opts, int nworkers,
                                 qtt_tensor** x, qtt_solve_info* info, void* stream) {
  try {
    QTT_REQUIRE(count >= 0 && K && f && opts && x, "qtt_solve_batched: null argument");
    if (count == 0) return QTT_OK;
    int dev = 0;
    QTT_CUDA(cudaGetDevice(&dev));
    const int W = std::max(1, std::min(nworkers > 0 ? nworkers : 8, count));
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    // Streams and events are released on every path, and the caller's
    // stream waits for every worker stream that was created, also when an
    // error ends the call early.
    struct Streams {
      cudaStream_t caller;
      cudaEvent_t ready = nullptr;
      std::vector<cudaStream_t> s;
      ~Streams() {
        for (cudaStream_t w : s) {
          cudaEvent_t done;
          if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
            if (cudaEventRecord(done, w) == cudaSuccess) cudaStreamWaitEvent(caller, done, 0);
            cudaEventDestroy(done);
          }
          cudaStreamDestroy(w);
        }
        if (ready) cudaEventDestroy(ready);
        cudaGetLastError();
      }
    } st{caller};
    // inputs may still be in flight on the caller's stream
    QTT_CUDA(cudaEventCreateWithFlags(&st.ready, cudaEventDisableTiming));
    QTT_CUDA(cudaEventRecord(st.ready, caller));
    std::vector<cudaStream_t>& streams = st.s;
    for (int w = 0; w < W; ++w) {
      cudaStream_t ws;
      QTT_CUDA(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
      streams.push_back(ws);
      QTT_CUDA(cudaStreamWaitEvent(ws, st.ready, 0));
    }
    std::atomic<int> next{0};
    std::atomic<int> first_error{QTT_OK};
    std::mutex msg_mu;
    std::string first_msg;
    for (int i = 0; i < count; ++i) x[i] = nullptr;
    auto worker = [&](int w) {
      cudaSetDevice(dev);
      StreamScope scope_(streams[w]);
      set_gpu_share(W);
      for (;;) {
        const int i = next.fetch_add(1);
        if (i >= count) break;
        qtt_solve_info local{};
        qtt_solve_info* inf = info ? &info[i] : &local;
        try {
          int rc = solve(K[i], f[i], x0 ? x0[i] : nullptr, nullptr, opts, &x[i], inf, streams[w]);
          inf->status = rc;
        } catch (const QttError& e) {
          inf->status = e.code;
          int z = QTT_OK;
          if (first_error.compare_exchange_strong(z, e.code)) {
            std::lock_guard<std::mutex> lk(msg_mu);
            first_msg = e.what();
          }
        } catch (const std::exception& e) {
          inf->status = QTT_EINVAL;
          int z = QTT_OK;
          if (first_error.compare_exchange_strong(z, QTT_EINVAL)) {
            std::lock_guard<std::mutex> lk(msg_mu);
            first_msg = e.what();
          }
        }
      }
    };
    std::vector<std::thread> threads;
    for (int w = 0; w < W; ++w) threads.emplace_back(worker, w);
    for (auto& t : threads) t.join();
    // results belong to the caller's stream (the worker streams end with
    // this call, after the caller's stream has been made to wait on them)
    for (int i = 0; i < count; ++i)
      if (x[i]) x[i]->stream = caller;
    if (first_error.load() != QTT_OK) {
      set_last_error("qtt_solve_batched: " + first_msg);
      return first_error.load();
    }
    return QTT_OK;
  } catch (const QttError& e) {
    set_last_error(e.what());
    return e.code;
  }
}
