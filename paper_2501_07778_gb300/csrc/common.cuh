// Shared internals of the QTT engine: error handling, device scratch arena,
// the tensor object, and declarations of the dense kernels every stage uses.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/qtt.h"

namespace qtt {

// ---------------------------------------------------------------------------
// Errors: internal code throws QttError; the C ABI catches and returns codes.
// ---------------------------------------------------------------------------
struct QttError : public std::runtime_error {
  int code;
  QttError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);

#define QTT_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      throw ::qtt::QttError(e_ == cudaErrorMemoryAllocation ? QTT_ENOMEM : QTT_ECUDA, \
                            std::string(#call) + ": " + cudaGetErrorString(e_) +      \
                                " (" __FILE__ ":" + std::to_string(__LINE__) + ")"); \
    }                                                                               \
  } while (0)

// every kernel launch of the library is followed by this check, which also
// counts the launch (qtt_kernel_launches)
void count_launch();
// every device allocation of the library is counted (qtt_device_allocations)
void count_alloc();
#define QTT_CHECK_LAUNCH()       \
  do {                           \
    ::qtt::count_launch();       \
    QTT_CUDA(cudaGetLastError()); \
  } while (0)

// Per-kernel-class CUDA-event timing, active after qtt_profile_enable(1).
enum ProfClass { PROF_GEMM_F64 = 0, PROF_GEMM_F32 = 1, PROF_CORE_PRODUCT = 2, PROF_QR_PANEL = 3, PROF_JACOBI = 4,
                 PROF_LU_PANEL = 5, PROF_PERMUTE = 6, PROF_TO_FULL = 7, PROF_PCG = 8, PROF_JACOBI_F32 = 9,
                 PROF_TC_GEMM = 10, PROF_NCLASS = 11 };
struct ProfToken {
  int cls;
  cudaEvent_t ev;
};
bool prof_on();
ProfToken prof_begin(int cls, cudaStream_t s);
void prof_end(const ProfToken& t, cudaStream_t s, double flops, double bytes);

// Streaming multiprocessors of the current device (queried once per device).
int num_sms();
// Grid for a grid-strided loop over n elements: one thread per element, at
// most per_sm blocks per SM.
inline int grid_for_n(long long n, int per_sm, int block = 256) {
  const long long cap = (long long)num_sms() * per_sm;
  long long g = (n + block - 1) / block;
  return (int)(g < 1 ? 1 : (g < cap ? g : cap));
}

#define QTT_REQUIRE(cond, msg)                                             \
  do {                                                                     \
    if (!(cond)) throw ::qtt::QttError(QTT_EINVAL, std::string(msg));      \
  } while (0)

// ---------------------------------------------------------------------------
// Scratch arena: stream-ordered allocations released together.
// ---------------------------------------------------------------------------
class Arena {
 public:
  explicit Arena(cudaStream_t s) : stream_(s) {}
  ~Arena() { release(); }
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  void* raw(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    count_alloc();
    cudaError_t e = cudaMallocAsync(&p, bytes, stream_);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw QttError(QTT_ENOMEM, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
    }
    ptrs_.push_back(p);
    return p;
  }
  template <typename T>
  T* alloc(size_t n) { return static_cast<T*>(raw(n * sizeof(T))); }
  void release() {
    for (void* p : ptrs_) cudaFreeAsync(p, stream_);
    ptrs_.clear();
  }
  cudaStream_t stream() const { return stream_; }

 private:
  cudaStream_t stream_;
  std::vector<void*> ptrs_;
};

}  // namespace qtt

namespace qtt {
// The finite-element problem an assembled stiffness MPO represents (set by
// qtt_assemble_stiffness, dropped when the MPO is changed in place): enough
// to apply the same operator as a stencil in full format (fe_residual.cu).
struct FeOperator {
  int L = 0, q = 0;
  std::vector<int> patch_xy;   // 2q integer patch offsets
  std::vector<int> bc;         // 4q side flags (left, right, bottom, top)
  double E = 0, nu = 0, gamma = 0;
};
}  // namespace qtt

// ---------------------------------------------------------------------------
// Tensor object (opaque to C callers).
// ---------------------------------------------------------------------------
struct qtt_tensor {
  int d = 0;
  int is_matrix = 0;
  int prec = QTT_F64;
  int n[QTT_MAX_CORES] = {0};
  int m[QTT_MAX_CORES] = {0};
  int r[QTT_MAX_CORES + 1] = {0};
  void* core[QTT_MAX_CORES] = {nullptr};
  size_t cap[QTT_MAX_CORES] = {0};   // elements allocated per core
  cudaStream_t stream = nullptr;     // stream the cores were allocated on (stream-ordered frees)
  int sym = 0;                       // MPO known to be symmetric (set by the assembly for q = 1)
  std::shared_ptr<const qtt::FeOperator> fe;   // assembled problem (stiffness MPOs only)
};

namespace qtt {

inline size_t esize(int prec) { return prec == QTT_F32 ? 4 : 8; }
inline size_t core_elems(const qtt_tensor* t, int k) {
  return (size_t)t->r[k] * t->n[k] * t->m[k] * t->r[k + 1];
}

// Tensor cores come from the stream-ordered allocator on the calling
// thread's current entry-point stream (set by StreamScope), so that freeing
// a temporary never synchronises the device.
cudaStream_t alloc_stream();
struct StreamScope {
  cudaStream_t prev;
  explicit StreamScope(cudaStream_t s);
  ~StreamScope();
};

qtt_tensor* tensor_alloc(int d, const int* n, const int* m, const int* r, int prec, int is_matrix);
void tensor_free(qtt_tensor* t);
// Make sure core k can hold `elems` elements (reallocates, discarding content).
void tensor_reserve(qtt_tensor* t, int k, size_t elems, cudaStream_t s);
qtt_tensor* tensor_clone(const qtt_tensor* src, int prec, cudaStream_t s);

// ---------------------------------------------------------------------------
// Dense kernels (column-major).  All are asynchronous on `s`.
// ---------------------------------------------------------------------------
// C = alpha op(A) op(B) + beta C, strided batch.
template <typename T>
void gemm(cudaStream_t s, bool tA, bool tB, int M, int N, int K, T alpha, const T* A, int lda,
          long long sA, const T* B, int ldb, long long sB, T beta, T* C, int ldc, long long sC,
          int batch = 1);

// out = permutation of a column-major tensor: out dim k is input dim perm[k].
template <typename T>
void permute(cudaStream_t s, const T* in, T* out, int nd, const int* dims, const int* perm, T alpha = T(1),
             T beta = T(0));

template <typename T>
void fill(cudaStream_t s, T* p, size_t n, T v);

// y = a x + b y
template <typename T>
void axpby(cudaStream_t s, size_t n, T a, const T* x, T b, T* y);

// strided 2D copy: dst[i + j ldd] = src[i + j lds], i < rows, j < cols
template <typename T>
void copy2d(cudaStream_t s, int rows, int cols, const T* src, int lds, T* dst, int ldd);

// convert precision
template <typename S, typename D>
void convert(cudaStream_t s, const S* src, D* dst, size_t n);

// out[0] = sum x^2 (device scalar, accumulated in double)
template <typename T>
void sumsq(cudaStream_t s, const T* x, size_t n, double* out);
// out[0] = sum x*y (device, double accumulation)
template <typename T>
void dotp(cudaStream_t s, const T* x, const T* y, size_t n, double* out);

// Einstein-summation contraction of two dense column-major operands
// (first index fastest), e.g. "aib,bBd->aiBd".  Labels are single chars;
// an index in both inputs but not in the output is summed; an index in both
// inputs and the output is a batch index.  C = alpha A*B + beta C.
template <typename T>
void einsum(cudaStream_t s, Arena& ar, const char* spec, const T* A, const int* dA, const T* B, const int* dB,
            T* C, T alpha = T(1), T beta = T(0));

// ---------------------------------------------------------------------------
// Dense factorizations (column-major).
// ---------------------------------------------------------------------------
// Householder QR of the m x n matrix A (lda): on return Q (m x k, ldq) and R
// (k x n, ldr) with k = min(m, n).  A is destroyed.
template <typename T>
void qr(cudaStream_t s, Arena& ar, int m, int n, T* A, int lda, T* Q, int ldq, T* R, int ldr);

// Thin SVD of the m x n matrix A: U (m x k), S (k), Vt (k x n), k = min(m,n),
// singular values descending.  A is destroyed.
template <typename T>
void svd(cudaStream_t s, Arena& ar, int m, int n, T* A, int lda, T* U, int ldu, T* S, T* Vt, int ldvt);

// Solve A X = B (A n x n, B n x nrhs) by LU with partial pivoting.  A and B
// are overwritten (B holds X).  Returns nonzero info on device in *info if a
// pivot is exactly zero.
template <typename T>
void lu_solve(cudaStream_t s, Arena& ar, int n, T* A, int lda, T* B, int ldb, int nrhs, int* info);

}  // namespace qtt
