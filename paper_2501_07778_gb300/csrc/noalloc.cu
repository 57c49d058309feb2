// qtt_to_full_noalloc: the Z-block expansion of a QTT vector (the same
// split into a left and a right partial expansion and the same GEMM chain as
// qtt_to_full) with the partial expansions kept in one fixed device buffer
// that is part of the library image instead of memory taken per call.
//
// Who needs this: code that must not allocate device memory while it runs,
// e.g. a caller inside a region where the allocator may not be entered (a
// real-time or signal-driven consumer, a host callback, a process that has
// pinned its memory budget up front), or a tool that must not perturb the
// allocator state it is inspecting.  qtt_to_full takes its temporaries from
// the stream-ordered pool and cannot serve them.
//
// Rules that follow from the one shared buffer:
//  * The first call on a device looks the buffer up (cudaGetSymbolAddress,
//    which may load the module); make it before any stream capture.
//  * Calls that overlap in time on one device (two streams, two threads)
//    share the buffer and race; the caller serialises them.
//  * Nothing in the buffer has to start at zero: every partial expansion is
//    written in full by its GEMM before it is read.
//  * Tensors whose partial expansions need more than the buffer holds are
//    rejected with QTT_EINVAL before anything is launched.
#include <mutex>
#include <string>

#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_full_scratch[kScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Address of this device's copy of the buffer; looked up once per device
// with that device current.
void* device_scratch() {
  int dev = 0;
  QTT_CUDA(cudaGetDevice(&dev));
  QTT_REQUIRE(dev >= 0 && dev < kMaxDevices, "qtt_to_full_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_full_scratch);
    // clear the runtime's sticky last-error slot so that the next library
    // call does not report this failure as its own
    if (e != cudaSuccess) cudaGetLastError();
    if (e != cudaSuccess || p == nullptr)
      throw qtt::QttError(QTT_ECUDA, std::string("qtt_to_full_noalloc: scratch lookup failed: ") +
                                         cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

size_t padded(long long elems, size_t esz) { return ((size_t)elems * esz + kAlign - 1) / kAlign * kAlign; }

template <typename T>
void expand_into(cudaStream_t s, const qtt_tensor* x, T* dst, unsigned char* scratch) {
  const int d = x->d;
  std::vector<long long> N(d);
  long long total = 1;
  for (int k = 0; k < d; ++k) {
    N[k] = x->n[k];
    total *= N[k];
  }
  if (d == 1) {
    QTT_CUDA(cudaMemcpyAsync(dst, x->core[0], sizeof(T) * N[0], cudaMemcpyDeviceToDevice, s));
    return;
  }
  int split = 1;
  long long left = N[0];
  while (split < d - 1 && left * left < total) {
    left *= N[split];
    ++split;
  }
  // plan every partial expansion's place in the buffer before launching
  std::vector<size_t> off_left(d, 0), off_right(d, 0);
  size_t used = 0;
  long long NL = N[0];
  for (int k = 1; k < split; ++k) {
    NL *= N[k];
    off_left[k] = used;
    used += padded(NL * x->r[k + 1], sizeof(T));
  }
  long long NR = N[d - 1];
  for (int k = d - 2; k >= split; --k) {
    NR *= N[k];
    off_right[k] = used;
    used += padded((long long)x->r[k] * NR, sizeof(T));
  }
  if (used > kScratchBytes)
    throw qtt::QttError(QTT_EINVAL, "qtt_to_full_noalloc: the partial expansions need " + std::to_string(used) +
                                        " bytes of scratch, above the fixed " + std::to_string(kScratchBytes) +
                                        "-byte buffer");
  QTT_REQUIRE(NL <= 2147483647LL && NR <= 2147483647LL, "qtt_to_full_noalloc: tensor too large");

  const T* PL = (const T*)x->core[0];
  NL = N[0];
  for (int k = 1; k < split; ++k) {
    T* out = reinterpret_cast<T*>(scratch + off_left[k]);
    qtt::gemm<T>(s, false, false, (int)NL, (int)(N[k] * x->r[k + 1]), x->r[k], T(1), PL, (int)NL, 0,
                 (const T*)x->core[k], x->r[k], 0, T(0), out, (int)NL, 0);
    PL = out;
    NL *= N[k];
  }
  const T* PR = (const T*)x->core[d - 1];
  NR = N[d - 1];
  for (int k = d - 2; k >= split; --k) {
    T* out = reinterpret_cast<T*>(scratch + off_right[k]);
    qtt::gemm<T>(s, false, false, (int)(x->r[k] * N[k]), (int)NR, x->r[k + 1], T(1), (const T*)x->core[k],
                 (int)(x->r[k] * N[k]), 0, PR, x->r[k + 1], 0, T(0), out, (int)(x->r[k] * N[k]), 0);
    PR = out;
    NR *= N[k];
  }
  qtt::gemm<T>(s, false, false, (int)NL, (int)NR, x->r[split], T(1), PL, (int)NL, 0, PR, x->r[split], 0, T(0), dst,
               (int)NL, 0);
}

}  // namespace

extern "C" int qtt_to_full_noalloc(const qtt_tensor* x, void* dst, size_t n_elems, void* stream) {
  try {
    QTT_REQUIRE(x && dst, "qtt_to_full_noalloc: null argument");
    QTT_REQUIRE(!x->is_matrix, "qtt_to_full_noalloc: only QTT vectors (MPS) are supported");
    long long total = 1;
    for (int k = 0; k < x->d; ++k) total *= (long long)x->n[k];
    QTT_REQUIRE((long long)n_elems == total, "qtt_to_full_noalloc: n_elems does not match the tensor size");
    unsigned char* scratch = static_cast<unsigned char*>(device_scratch());
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (x->prec == QTT_F64) expand_into<double>(s, x, (double*)dst, scratch);
    else expand_into<float>(s, x, (float*)dst, scratch);
    return QTT_OK;
  } catch (const qtt::QttError& e) {
    qtt::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    qtt::set_last_error(e.what());
    return QTT_EINVAL;
  }
}
