// extern "C" entry points: argument checking, precision dispatch, and the
// translation of internal exceptions into QTT_E* codes.
#include <cmath>
#include <cstring>
#include <string>

#include "common.cuh"
#include "tt_ops.cuh"

namespace qtt {
namespace {
thread_local std::string g_last_error;
}
double residual64(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f);
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace qtt

using namespace qtt;

#define QTT_API_BEGIN try {
#define QTT_API_END                                      \
  }                                                      \
  catch (const QttError& e) {                            \
    set_last_error(e.what());                            \
    return e.code;                                       \
  }                                                      \
  catch (const std::exception& e) {                      \
    set_last_error(e.what());                            \
    return QTT_EINVAL;                                   \
  }                                                      \
  catch (...) {                                          \
    set_last_error("unknown error");                     \
    return QTT_EINVAL;                                   \
  }

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

const char* qtt_last_error(void) { return g_last_error.c_str(); }

int qtt_tensor_create(int d, const int* n, const int* m, const int* ranks, int prec, const void* const* host_cores,
                      qtt_tensor** out) {
  QTT_API_BEGIN
  QTT_REQUIRE(out && n && ranks && host_cores, "qtt_tensor_create: null argument");
  bool is_matrix = false;
  if (m)
    for (int k = 0; k < d; ++k) is_matrix = is_matrix || (m[k] != 1);
  qtt_tensor* t = tensor_alloc(d, n, m, ranks, prec, m != nullptr && is_matrix ? 1 : 0);
  if (m && !is_matrix) t->is_matrix = 0;
  try {
    for (int k = 0; k < d; ++k) {
      QTT_REQUIRE(host_cores[k] != nullptr, "qtt_tensor_create: null core");
      QTT_CUDA(cudaMemcpy(t->core[k], host_cores[k], core_elems(t, k) * esize(prec), cudaMemcpyHostToDevice));
    }
  } catch (...) {
    tensor_free(t);
    throw;
  }
  *out = t;
  return QTT_OK;
  QTT_API_END
}

int qtt_tensor_info(const qtt_tensor* t, int* d, int* n, int* m, int* ranks, int* prec) {
  QTT_API_BEGIN
  QTT_REQUIRE(t, "qtt_tensor_info: null tensor");
  if (d) *d = t->d;
  if (prec) *prec = t->prec;
  for (int k = 0; k < t->d; ++k) {
    if (n) n[k] = t->n[k];
    if (m) m[k] = t->m[k];
  }
  if (ranks)
    for (int k = 0; k <= t->d; ++k) ranks[k] = t->r[k];
  return QTT_OK;
  QTT_API_END
}

int qtt_tensor_get_cores(const qtt_tensor* t, void* const* host_dst) {
  QTT_API_BEGIN
  QTT_REQUIRE(t && host_dst, "qtt_tensor_get_cores: null argument");
  QTT_CUDA(cudaDeviceSynchronize());
  for (int k = 0; k < t->d; ++k)
    QTT_CUDA(cudaMemcpy(host_dst[k], t->core[k], core_elems(t, k) * esize(t->prec), cudaMemcpyDeviceToHost));
  return QTT_OK;
  QTT_API_END
}

int qtt_tensor_core_ptr(const qtt_tensor* t, int k, void** dev_ptr) {
  QTT_API_BEGIN
  QTT_REQUIRE(t && dev_ptr && k >= 0 && k < t->d, "qtt_tensor_core_ptr: bad argument");
  *dev_ptr = t->core[k];
  return QTT_OK;
  QTT_API_END
}

int qtt_tensor_copy(const qtt_tensor* src, int prec, qtt_tensor** out, void* stream) {
  QTT_API_BEGIN
  QTT_REQUIRE(src && out, "qtt_tensor_copy: null argument");
  StreamScope scope_(as_stream(stream));
  *out = tensor_clone(src, prec, as_stream(stream));
  return QTT_OK;
  QTT_API_END
}

void qtt_free(qtt_tensor* t) { tensor_free(t); }

int qtt_to_full(const qtt_tensor* x, void* dst, size_t n_elems, int ordering, void* stream) {
  QTT_API_BEGIN
  QTT_REQUIRE(x && dst, "qtt_to_full: null argument");
  cudaStream_t s = as_stream(stream);
  StreamScope scope_(s);
  Arena ar(s);
  if (x->prec == QTT_F64) to_full<double>(s, ar, x, (double*)dst, n_elems, ordering);
  else to_full<float>(s, ar, x, (float*)dst, n_elems, ordering);
  return QTT_OK;
  QTT_API_END
}

int qtt_round(qtt_tensor* x, double tol, int max_rank, void* stream) {
  QTT_API_BEGIN
  QTT_REQUIRE(x, "qtt_round: null tensor");
  QTT_REQUIRE(tol >= 0.0, "qtt_round: negative tolerance");
  x->fe.reset();   // rounded in place: no longer the assembled operator exactly
  cudaStream_t s = as_stream(stream);
  StreamScope scope_(s);
  Arena ar(s);
  int rc = x->prec == QTT_F64 ? round_tt<double>(s, ar, x, tol, max_rank) : round_tt<float>(s, ar, x, tol, max_rank);
  QTT_CUDA(cudaStreamSynchronize(s));
  if (rc != QTT_OK) set_last_error("qtt_round: rank cap reached");
  return rc;
  QTT_API_END
}

int qtt_matvec(const qtt_tensor* A, const qtt_tensor* x, double tol, int max_rank, qtt_tensor** y, void* stream) {
  QTT_API_BEGIN
  QTT_REQUIRE(A && x && y, "qtt_matvec: null argument");
  cudaStream_t s = as_stream(stream);
  StreamScope scope_(s);
  qtt_tensor* out = A->prec == QTT_F64 ? product<double>(s, A, x) : product<float>(s, A, x);
  int rc = QTT_OK;
  if (tol > 0.0) {
    try {
      Arena ar(s);
      rc = out->prec == QTT_F64 ? round_tt<double>(s, ar, out, tol, max_rank)
                                : round_tt<float>(s, ar, out, tol, max_rank);
    } catch (...) {
      tensor_free(out);
      throw;
    }
  }
  *y = out;
  return rc;
  QTT_API_END
}

int qtt_axpby(double alpha, const qtt_tensor* x, double beta, const qtt_tensor* y, qtt_tensor** z, void* stream) {
  QTT_API_BEGIN
  QTT_REQUIRE(x && y && z, "qtt_axpby: null argument");
  cudaStream_t s = as_stream(stream);
  StreamScope scope_(s);
  *z = x->prec == QTT_F64 ? tt_sum<double>(s, alpha, x, beta, y) : tt_sum<float>(s, (float)alpha, x, (float)beta, y);
  return QTT_OK;
  QTT_API_END
}

int qtt_norm(const qtt_tensor* x, double* out, void* stream) {
  QTT_API_BEGIN
  QTT_REQUIRE(x && out, "qtt_norm: null argument");
  cudaStream_t s = as_stream(stream);
  StreamScope scope_(s);
  Arena ar(s);
  *out = x->prec == QTT_F64 ? norm<double>(s, ar, x) : norm<float>(s, ar, x);
  return QTT_OK;
  QTT_API_END
}

int qtt_residual(const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f, double* out, void* stream) {
  QTT_API_BEGIN
  QTT_REQUIRE(K && u && f && out, "qtt_residual: null argument");
  QTT_REQUIRE(K->prec == QTT_F64 && u->prec == QTT_F64 && f->prec == QTT_F64, "qtt_residual: operands must be FP64");
  QTT_REQUIRE(K->is_matrix && !u->is_matrix && !f->is_matrix && K->d == u->d && K->d == f->d,
              "qtt_residual: K must be an MPO and u, f MPS of equal length");
  cudaStream_t s = as_stream(stream);
  StreamScope scope_(s);
  *out = residual64(s, K, u, f);
  return QTT_OK;
  QTT_API_END
}

int qtt_round_residual(const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f, int rank,
                       unsigned long long seed, double* kept_norm, qtt_tensor** r, void* stream) {
  QTT_API_BEGIN
  QTT_REQUIRE(K && u && f && r, "qtt_round_residual: null argument");
  QTT_REQUIRE(K->d >= 2, "qtt_round_residual: needs at least two cores");
  cudaStream_t s = as_stream(stream);
  StreamScope scope_(s);
  *r = round_residual_rand(s, K, u, f, rank, seed, kept_norm);
  return QTT_OK;
  QTT_API_END
}

}  // extern "C"
