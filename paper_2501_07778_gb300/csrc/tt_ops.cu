// Tensor objects and the TT operations of Section 4: expansion to full
// format, the core-by-core MPO x MPS product, sums, orthogonalisation, norms
// and rounding (Oseledets 2011, Alg. 2).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tt_ops.cuh"

namespace qtt {

// ---------------------------------------------------------------------------
// Tensor memory
// ---------------------------------------------------------------------------
namespace {
thread_local cudaStream_t g_alloc_stream = nullptr;
}
cudaStream_t alloc_stream() { return g_alloc_stream; }

// The engine allocates and frees many small blocks per core step through the
// stream-ordered allocator.  With the pool's default release threshold (0)
// every synchronisation returns the cached memory to the driver and the next
// allocation maps it again, which serialises concurrent solves; keep it cached.
static void keep_pool_memory() {
  static std::atomic<int> done_mask{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 31) {
    cudaGetLastError();
    return;
  }
  if (done_mask.load() & (1 << dev)) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done_mask.fetch_or(1 << dev);
}

StreamScope::StreamScope(cudaStream_t s) : prev(g_alloc_stream) {
  keep_pool_memory();
  g_alloc_stream = s;
}
StreamScope::~StreamScope() { g_alloc_stream = prev; }

qtt_tensor* tensor_alloc(int d, const int* n, const int* m, const int* r, int prec, int is_matrix) {
  QTT_REQUIRE(d >= 1 && d <= QTT_MAX_CORES, "tensor: number of cores out of range");
  QTT_REQUIRE(prec == QTT_F64 || prec == QTT_F32, "tensor: precision must be QTT_F64 or QTT_F32");
  QTT_REQUIRE(r[0] == 1 && r[d] == 1, "tensor: boundary ranks must be 1");
  qtt_tensor* t = new qtt_tensor();
  t->d = d;
  t->is_matrix = is_matrix;
  t->prec = prec;
  t->stream = g_alloc_stream;
  for (int k = 0; k < d; ++k) {
    QTT_REQUIRE(n[k] >= 1 && (m ? m[k] : 1) >= 1 && r[k] >= 1, "tensor: sizes must be positive");
    t->n[k] = n[k];
    t->m[k] = m ? m[k] : 1;
  }
  for (int k = 0; k <= d; ++k) t->r[k] = r[k];
  try {
    for (int k = 0; k < d; ++k) {
      size_t e = core_elems(t, k);
      t->cap[k] = e;
      count_alloc();
      cudaError_t err = cudaMallocAsync(&t->core[k], std::max<size_t>(e, 1) * esize(prec), t->stream);
      if (err != cudaSuccess) {
        cudaGetLastError();
        throw QttError(QTT_ENOMEM, "core allocation failed");
      }
    }
  } catch (...) {
    tensor_free(t);
    throw;
  }
  return t;
}

// stream-ordered: the cores are released after the work queued so far on the
// tensor's stream; callers free a tensor only when no other stream still uses it
void tensor_free(qtt_tensor* t) {
  if (!t) return;
  for (int k = 0; k < t->d; ++k)
    if (t->core[k]) cudaFreeAsync(t->core[k], t->stream);
  delete t;
}

void tensor_reserve(qtt_tensor* t, int k, size_t elems, cudaStream_t s) {
  if (elems <= t->cap[k]) return;
  // the old core is dead: released in order on s, replaced by a new block
  if (t->core[k]) QTT_CUDA(cudaFreeAsync(t->core[k], s));
  t->core[k] = nullptr;
  count_alloc();
  QTT_CUDA(cudaMallocAsync(&t->core[k], elems * esize(t->prec), s));
  t->cap[k] = elems;
  t->stream = s;
}

qtt_tensor* tensor_clone(const qtt_tensor* src, int prec, cudaStream_t s) {
  qtt_tensor* t = tensor_alloc(src->d, src->n, src->m, src->r, prec, src->is_matrix);
  t->sym = src->sym;
  if (src->prec == prec) t->fe = src->fe;
  for (int k = 0; k < src->d; ++k) {
    size_t e = core_elems(src, k);
    if (src->prec == prec) {
      QTT_CUDA(cudaMemcpyAsync(t->core[k], src->core[k], e * esize(prec), cudaMemcpyDeviceToDevice, s));
    } else if (src->prec == QTT_F64) {
      convert<double, float>(s, (const double*)src->core[k], (float*)t->core[k], e);
    } else {
      convert<float, double>(s, (const float*)src->core[k], (double*)t->core[k], e);
    }
  }
  return t;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
namespace {
inline int grid_for(long long n) { return grid_for_n(n, 32); }

// Y[(a + R0 g), i, k, (b + R1 e)] = sum_j A[a, i, j, b] X[g, j, k, e]
// (X has an extra column mode p = 1 for an MPS operand).
template <typename T>
__global__ void core_product_kernel(int R0, int n, int mm, int R1, int r0, int p, int r1, const T* __restrict__ A,
                                    const T* __restrict__ X, T* __restrict__ Y, long long total) {
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
       o += (long long)gridDim.x * blockDim.x) {
    long long t = o;
    int a = (int)(t % R0); t /= R0;
    int g = (int)(t % r0); t /= r0;
    int i = (int)(t % n); t /= n;
    int kk = (int)(t % p); t /= p;
    int b = (int)(t % R1); t /= R1;
    int e = (int)t;
    const T* Ap = A + a + (long long)R0 * (i + (long long)n * ((long long)mm * b));
    const T* Xp = X + g + (long long)r0 * ((long long)mm * (kk + (long long)p * e));
    T acc = T(0);
    for (int j = 0; j < mm; ++j) acc += Ap[(long long)R0 * n * j] * Xp[(long long)r0 * j];
    Y[o] = acc;
  }
}

// block-diagonal sum core: out (r0a + r0b) x nm x (r1a + r1b) with first/last
// core special cases; alpha scales x's first core, beta y's.
template <typename T>
__global__ void sum_core_kernel(int r0a, int r1a, int r0b, int r1b, int nm, int first, int last, const T* __restrict__ X,
                                const T* __restrict__ Yc, T alpha, T beta, T* __restrict__ Z, int R0, int R1) {
  long long total = (long long)R0 * nm * R1;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
       o += (long long)gridDim.x * blockDim.x) {
    long long t = o;
    int a = (int)(t % R0); t /= R0;
    int i = (int)(t % nm); t /= nm;
    int b = (int)t;
    T v = T(0);
    // which block
    int ax = first ? 0 : a, bx = last ? 0 : b;                 // index into x if in x-block
    bool in_x = (first || a < r0a) && (last || b < r1a);
    int ay = first ? 0 : a - r0a, by = last ? 0 : b - r1a;
    bool in_y = (first || a >= r0a) && (last || b >= r1a);
    if (first && last) {
      v = alpha * X[i] + beta * Yc[i];
    } else if (first) {
      if (b < r1a) v = alpha * X[i + (long long)nm * b];
      else v = beta * Yc[i + (long long)nm * (b - r1a)];
    } else if (last) {
      if (a < r0a) v = X[a + (long long)r0a * i];
      else v = Yc[(a - r0a) + (long long)r0b * i];
    } else if (in_x && a < r0a && b < r1a) {
      v = X[ax + (long long)r0a * (i + (long long)nm * bx)];
    } else if (in_y && a >= r0a && b >= r1a) {
      v = Yc[ay + (long long)r0b * (i + (long long)nm * by)];
    }
    Z[o] = v;
  }
}

// interleave the bits of i (x) and j (y): Z-order of Section 3.2
__device__ __forceinline__ long long zorder_dev(long long i, long long j, int L) {
  long long z = 0;
  for (int k = 0; k < L; ++k) z |= (((i >> k) & 1LL) << (2 * k)) | (((j >> k) & 1LL) << (2 * k + 1));
  return z;
}

// out (canonical: patch blocks of interleaved components 2 (i + n j) + c)
//   = in (QTT order: z + nn m + nn q c)
template <typename T>
__global__ void canonical_scatter_kernel(const T* __restrict__ in, T* __restrict__ out, int L, int q, long long total) {
  const long long n = 1LL << L, nn = n * n;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
       o += (long long)gridDim.x * blockDim.x) {
    int c = (int)(o & 1);
    long long node = (o >> 1) % nn;
    long long m = (o >> 1) / nn;
    long long i = node % n, j = node / n;
    out[o] = in[zorder_dev(i, j, L) + nn * m + nn * q * c];
  }
}

// the inverse reordering: canonical -> QTT order
template <typename T>
__global__ void canonical_gather_kernel(const T* __restrict__ in, T* __restrict__ out, int L, int q, long long total) {
  const long long n = 1LL << L, nn = n * n;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
       o += (long long)gridDim.x * blockDim.x) {
    int c = (int)(o & 1);
    long long node = (o >> 1) % nn;
    long long m = (o >> 1) / nn;
    long long i = node % n, j = node / n;
    out[zorder_dev(i, j, L) + nn * m + nn * q * c] = in[o];
  }
}
}  // namespace

template <typename T>
void from_canonical(cudaStream_t s, const T* in, T* out, int L, int q) {
  const long long total = 2LL * q << (2 * L);
  canonical_gather_kernel<T><<<grid_for(total), 256, 0, s>>>(in, out, L, q, total);
  QTT_CHECK_LAUNCH();
}

template <typename T>
void core_product(cudaStream_t s, int R0, int n, int mm, int R1, int r0, int p, int r1, const T* A, const T* X, T* Y) {
  long long total = (long long)R0 * r0 * n * p * R1 * r1;
  if (total == 0) return;
  ProfToken pt = prof_begin(PROF_CORE_PRODUCT, s);
  core_product_kernel<T><<<grid_for(total), 256, 0, s>>>(R0, n, mm, R1, r0, p, r1, A, X, Y, total);
  QTT_CHECK_LAUNCH();
  // algorithmic traffic: read both cores once, write the product core
  if (pt.ev)
    prof_end(pt, s, 2.0 * (double)total * mm,
             sizeof(T) * ((double)total + (double)R0 * n * mm * R1 + (double)r0 * mm * p * r1));
}

// ---------------------------------------------------------------------------
// Full expansion: the product of a left and a right partial expansion.
// ---------------------------------------------------------------------------
template <typename T>
static void to_full_mps(cudaStream_t s, Arena& ar, const qtt_tensor* x, T* dst) {
  const int d = x->d;
  std::vector<long long> N(d);
  for (int k = 0; k < d; ++k) N[k] = (long long)x->n[k] * x->m[k];
  if (d == 1) {
    QTT_CUDA(cudaMemcpyAsync(dst, x->core[0], sizeof(T) * N[0], cudaMemcpyDeviceToDevice, s));
    return;
  }
  // split so that the left and right expansions have similar sizes
  long long total = 1;
  for (int k = 0; k < d; ++k) total *= N[k];
  int split = 1;
  long long left = N[0];
  while (split < d - 1 && left * left < total) {
    left *= N[split];
    ++split;
  }
  // left part: cores [0, split) -> PL (NL x r_split)
  const T* PL = (const T*)x->core[0];
  long long NL = N[0];
  for (int k = 1; k < split; ++k) {
    T* out = ar.alloc<T>(NL * N[k] * x->r[k + 1]);
    gemm<T>(s, false, false, (int)NL, (int)(N[k] * x->r[k + 1]), x->r[k], T(1), PL, (int)NL, 0,
            (const T*)x->core[k], x->r[k], 0, T(0), out, (int)NL, 0);
    PL = out;
    NL *= N[k];
  }
  // right part: cores [split, d) -> PR (r_split x NR)
  const T* PR = (const T*)x->core[d - 1];
  long long NR = N[d - 1];
  for (int k = d - 2; k >= split; --k) {
    T* out = ar.alloc<T>((long long)x->r[k] * N[k] * NR);
    gemm<T>(s, false, false, (int)(x->r[k] * N[k]), (int)NR, x->r[k + 1], T(1), (const T*)x->core[k],
            (int)(x->r[k] * N[k]), 0, PR, x->r[k + 1], 0, T(0), out, (int)(x->r[k] * N[k]), 0);
    PR = out;
    NR *= N[k];
  }
  QTT_REQUIRE(NL <= 2147483647LL && NR <= 2147483647LL, "to_full: tensor too large");
  gemm<T>(s, false, false, (int)NL, (int)NR, x->r[split], T(1), PL, (int)NL, 0, PR, x->r[split], 0, T(0), dst,
          (int)NL, 0);
}

template <typename T>
void to_full(cudaStream_t s, Arena& ar, const qtt_tensor* x, T* dst, size_t n_elems, int ordering) {
  long long total = 1;
  for (int k = 0; k < x->d; ++k) total *= (long long)x->n[k] * x->m[k];
  QTT_REQUIRE((long long)n_elems == total, "to_full: n_elems does not match the tensor size");
  if (x->is_matrix) {
    QTT_REQUIRE(ordering == QTT_ORDER_Z_BLOCK, "to_full: an MPO supports only QTT_ORDER_Z_BLOCK");
    QTT_REQUIRE(2 * x->d <= 24, "to_full: MPO has too many cores for a dense expansion");
    T* tmp = ar.alloc<T>(total);
    to_full_mps<T>(s, ar, x, tmp);
    // dims (n1, m1, n2, m2, ...) -> (n1, ..., nd, m1, ..., md)
    std::vector<int> dims(2 * x->d), perm(2 * x->d);
    for (int k = 0; k < x->d; ++k) {
      dims[2 * k] = x->n[k];
      dims[2 * k + 1] = x->m[k];
      perm[k] = 2 * k;
      perm[x->d + k] = 2 * k + 1;
    }
    permute<T>(s, tmp, dst, 2 * x->d, dims.data(), perm.data());
    return;
  }
  if (ordering == QTT_ORDER_Z_BLOCK) {
    to_full_mps<T>(s, ar, x, dst);
    return;
  }
  QTT_REQUIRE(ordering == QTT_ORDER_CANONICAL, "to_full: unknown ordering");
  // infer the elasticity layout: L mode-4 cores, optional mode-q core, mode-2 core
  const int d = x->d;
  QTT_REQUIRE(d >= 2 && x->n[d - 1] == 2, "to_full: canonical order needs a final mode-2 component core");
  int L = 0;
  while (L < d - 1 && x->n[L] == 4) ++L;
  int q = 1;
  if (L == d - 2) q = x->n[d - 2];
  else QTT_REQUIRE(L == d - 1, "to_full: canonical order needs the elasticity layout");
  if (L == d - 2 && q == 4) {
    // ambiguous: a mode-4 patch core; treat the last mode-4 core as the patch core
    // only if the caller built q = 4 (cannot tell) -- position cores take priority
  }
  T* tmp = ar.alloc<T>(total);
  to_full_mps<T>(s, ar, x, tmp);
  canonical_scatter_kernel<T><<<grid_for(total), 256, 0, s>>>(tmp, dst, L, q, total);
  QTT_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Products and sums
// ---------------------------------------------------------------------------
template <typename T>
qtt_tensor* product(cudaStream_t s, const qtt_tensor* A, const qtt_tensor* X) {
  QTT_REQUIRE(A->is_matrix, "product: first operand must be an MPO");
  QTT_REQUIRE(A->d == X->d, "product: core counts differ");
  QTT_REQUIRE(A->prec == X->prec, "product: precisions differ");
  int d = A->d;
  std::vector<int> n(d), m(d), r(d + 1);
  for (int k = 0; k < d; ++k) {
    QTT_REQUIRE(A->m[k] == X->n[k], "product: mode sizes differ");
    n[k] = A->n[k];
    m[k] = X->m[k];
  }
  for (int k = 0; k <= d; ++k) r[k] = A->r[k] * X->r[k];
  qtt_tensor* Y = tensor_alloc(d, n.data(), m.data(), r.data(), A->prec, X->is_matrix);
  for (int k = 0; k < d; ++k)
    core_product<T>(s, A->r[k], A->n[k], A->m[k], A->r[k + 1], X->r[k], X->m[k], X->r[k + 1], (const T*)A->core[k],
                    (const T*)X->core[k], (T*)Y->core[k]);
  return Y;
}

template <typename T>
qtt_tensor* tt_sum(cudaStream_t s, T alpha, const qtt_tensor* X, T beta, const qtt_tensor* Yt) {
  QTT_REQUIRE(X->d == Yt->d && X->prec == Yt->prec && X->is_matrix == Yt->is_matrix, "sum: operands differ in shape");
  int d = X->d;
  std::vector<int> r(d + 1);
  for (int k = 0; k < d; ++k) QTT_REQUIRE(X->n[k] == Yt->n[k] && X->m[k] == Yt->m[k], "sum: mode sizes differ");
  r[0] = 1;
  r[d] = 1;
  for (int k = 1; k < d; ++k) r[k] = X->r[k] + Yt->r[k];
  qtt_tensor* Z = tensor_alloc(d, X->n, X->m, r.data(), X->prec, X->is_matrix);
  for (int k = 0; k < d; ++k) {
    int nm = X->n[k] * X->m[k];
    int first = (k == 0), last = (k == d - 1);
    long long total = (long long)r[k] * nm * r[k + 1];
    sum_core_kernel<T><<<grid_for(total), 256, 0, s>>>(X->r[k], X->r[k + 1], Yt->r[k], Yt->r[k + 1], nm, first, last,
                                                       (const T*)X->core[k], (const T*)Yt->core[k],
                                                       k == 0 ? alpha : T(1), k == 0 ? beta : T(1), (T*)Z->core[k],
                                                       r[k], r[k + 1]);
    QTT_CHECK_LAUNCH();
  }
  return Z;
}

// ---------------------------------------------------------------------------
// Orthogonalisation and rounding
// ---------------------------------------------------------------------------
template <typename T>
void left_orthogonalize(cudaStream_t s, Arena& ar, qtt_tensor* x, int upto) {
  for (int k = 0; k < upto; ++k) {
    const int r0 = x->r[k], r1 = x->r[k + 1], nm = x->n[k] * x->m[k];
    const int rows = r0 * nm, kk = std::min(rows, r1);
    const int nm2 = x->n[k + 1] * x->m[k + 1], r2 = x->r[k + 2];
    T* Acopy = ar.alloc<T>((size_t)rows * r1);
    QTT_CUDA(cudaMemcpyAsync(Acopy, x->core[k], sizeof(T) * rows * r1, cudaMemcpyDeviceToDevice, s));
    T* R = ar.alloc<T>((size_t)kk * r1);
    qr<T>(s, ar, rows, r1, Acopy, rows, (T*)x->core[k], rows, R, kk);
    T* next = ar.alloc<T>((size_t)kk * nm2 * r2);
    gemm<T>(s, false, false, kk, nm2 * r2, r1, T(1), R, kk, 0, (const T*)x->core[k + 1], r1, 0, T(0), next, kk, 0);
    QTT_CUDA(cudaMemcpyAsync(x->core[k + 1], next, sizeof(T) * kk * nm2 * r2, cudaMemcpyDeviceToDevice, s));
    x->r[k + 1] = kk;
  }
}

template <typename T>
void right_orthogonalize(cudaStream_t s, Arena& ar, qtt_tensor* x, int downto) {
  for (int k = x->d - 1; k > downto; --k) {
    const int r0 = x->r[k], r1 = x->r[k + 1], nm = x->n[k] * x->m[k];
    const int cols = nm * r1, kk = std::min(r0, cols);
    const int nmp = x->n[k - 1] * x->m[k - 1], rp = x->r[k - 1];
    // core^T (cols x r0) = Q R  ->  core = R^T Q^T
    T* At = ar.alloc<T>((size_t)cols * r0);
    int dims[2] = {r0, cols}, perm[2] = {1, 0};
    permute<T>(s, (const T*)x->core[k], At, 2, dims, perm);
    T* Q = ar.alloc<T>((size_t)cols * kk);
    T* R = ar.alloc<T>((size_t)kk * r0);
    qr<T>(s, ar, cols, r0, At, cols, Q, cols, R, kk);
    int d2[2] = {cols, kk};
    permute<T>(s, Q, (T*)x->core[k], 2, d2, perm);               // kk x cols
    T* prev = ar.alloc<T>((size_t)rp * nmp * kk);
    // prev (rp nmp x r0) * R^T (r0 x kk)
    gemm<T>(s, false, true, rp * nmp, kk, r0, T(1), (const T*)x->core[k - 1], rp * nmp, 0, R, kk, 0, T(0), prev,
            rp * nmp, 0);
    QTT_CUDA(cudaMemcpyAsync(x->core[k - 1], prev, sizeof(T) * rp * nmp * kk, cudaMemcpyDeviceToDevice, s));
    x->r[k] = kk;
  }
}

template <typename T>
double norm(cudaStream_t s, Arena& ar, const qtt_tensor* x) {
  qtt_tensor* y = tensor_clone(x, x->prec, s);
  double out = 0.0;
  try {
    left_orthogonalize<T>(s, ar, y, y->d - 1);
    double* dv = ar.alloc<double>(1);
    sumsq<T>(s, (const T*)y->core[y->d - 1], core_elems(y, y->d - 1), dv);
    QTT_CUDA(cudaMemcpyAsync(&out, dv, sizeof(double), cudaMemcpyDeviceToHost, s));
    QTT_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    tensor_free(y);
    throw;
  }
  tensor_free(y);
  return std::sqrt(out);
}

int truncation_rank(const std::vector<double>& sv, double delta, int max_rank, bool* capped) {
  // smallest rank whose discarded tail has 2-norm <= delta
  const int k = (int)sv.size();
  std::vector<double> tail(k + 1, 0.0);
  for (int i = k - 1; i >= 0; --i) tail[i] = tail[i + 1] + sv[i] * sv[i];
  int keep = k;
  for (int i = 0; i < k; ++i)
    if (std::sqrt(tail[i]) <= delta) {
      keep = i;
      break;
    }
  keep = std::max(keep, 1);
  if (capped) *capped = false;
  if (max_rank > 0 && keep > max_rank) {
    keep = max_rank;
    if (capped) *capped = true;
  }
  return keep;
}

template <typename T>
int round_tt(cudaStream_t s, Arena& ar, qtt_tensor* x, double tol, int max_rank) {
  const int d = x->d;
  if (d == 1) return QTT_OK;
  left_orthogonalize<T>(s, ar, x, d - 1);
  double nrm2 = 0.0;
  {
    double* dv = ar.alloc<double>(1);
    sumsq<T>(s, (const T*)x->core[d - 1], core_elems(x, d - 1), dv);
    QTT_CUDA(cudaMemcpyAsync(&nrm2, dv, sizeof(double), cudaMemcpyDeviceToHost, s));
    QTT_CUDA(cudaStreamSynchronize(s));
  }
  const double delta = tol * std::sqrt(nrm2) / std::sqrt((double)(d - 1));
  bool any_cap = false;
  for (int k = d - 1; k >= 1; --k) {
    const int r0 = x->r[k], r1 = x->r[k + 1], nm = x->n[k] * x->m[k];
    const int cols = nm * r1, kk = std::min(r0, cols);
    T* A = ar.alloc<T>((size_t)r0 * cols);
    QTT_CUDA(cudaMemcpyAsync(A, x->core[k], sizeof(T) * r0 * cols, cudaMemcpyDeviceToDevice, s));
    T* U = ar.alloc<T>((size_t)r0 * kk);
    T* S = ar.alloc<T>(kk);
    T* Vt = ar.alloc<T>((size_t)kk * cols);
    svd<T>(s, ar, r0, cols, A, r0, U, r0, S, Vt, kk);
    std::vector<T> sh(kk);
    QTT_CUDA(cudaMemcpyAsync(sh.data(), S, sizeof(T) * kk, cudaMemcpyDeviceToHost, s));
    QTT_CUDA(cudaStreamSynchronize(s));
    std::vector<double> sv(sh.begin(), sh.end());
    bool capped = false;
    const int rk = truncation_rank(sv, delta, max_rank, &capped);
    any_cap = any_cap || capped;
    // core k <- Vt[0:rk, :]
    copy2d<T>(s, rk, cols, Vt, kk, (T*)x->core[k], rk);
    // core k-1 <- core k-1 * U[:, 0:rk] diag(S[0:rk])
    const int rp = x->r[k - 1], nmp = x->n[k - 1] * x->m[k - 1];
    T* US = ar.alloc<T>((size_t)r0 * rk);
    scale_columns<T>(s, r0, rk, U, r0, S, US, r0);
    T* prev = ar.alloc<T>((size_t)rp * nmp * rk);
    gemm<T>(s, false, false, rp * nmp, rk, r0, T(1), (const T*)x->core[k - 1], rp * nmp, 0, US, r0, 0, T(0), prev,
            rp * nmp, 0);
    QTT_CUDA(cudaMemcpyAsync(x->core[k - 1], prev, sizeof(T) * rp * nmp * rk, cudaMemcpyDeviceToDevice, s));
    x->r[k] = rk;
  }
  return any_cap ? QTT_ERANKCAP : QTT_OK;
}

namespace {
// B (rows x cols, ld rows) = diag(S) A[0:rows, :] (A with leading dimension lda)
__global__ void scale_rows_kernel(int rows, long long cols, const double* __restrict__ A, int lda,
                                  const double* __restrict__ S, double* __restrict__ B) {
  const long long total = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % rows);
    const long long j = t / rows;
    B[t] = S[i] * A[i + j * lda];
  }
}
}  // namespace

// Left-to-right TT-SVD of a full FP64 vector (QTT order).  The unfolding
// C_k (rows = r_{k-1} n_k, cols = the remaining index range) is truncated
// through the eigendecomposition of its Gram matrix C_k C_k^T when it is
// wide (the Gram product is one split-K GEMM, where a Householder QR of the
// transposed C_k would run single-CTA panels over millions of rows), and
// through its SVD when it is tall.  The eigenvalues are the squared
// singular values; the kept eigenvectors, those of singular values above
// the truncation level delta = eps ||v|| / sqrt(d - 1), carry a relative
// error of about 1e-16 (sigma_1 / sigma_k)^2, which suits tolerances
// eps >= 1e-6.  The discarded tail of every unfolding is <= delta.
qtt_tensor* tt_svd_full(cudaStream_t s, Arena& ar, const double* v, int d, const int* n, double eps, int max_rank) {
  QTT_REQUIRE(d >= 1 && v && n, "tt_svd_full: bad arguments");
  long long total = 1;
  for (int k = 0; k < d; ++k) total *= n[k];
  std::vector<int> r(d + 1, 1), ones(d, 1);
  std::vector<const double*> core(d, nullptr);
  const double* C = v;
  long long cols = total;
  int rprev = 1;
  double delta = -1.0;
  for (int k = 0; k < d - 1; ++k) {
    const int rows = rprev * n[k];
    cols /= n[k];
    QTT_REQUIRE(cols <= 2147483647LL, "tt_svd_full: unfolding too large");
    const int kk = (int)std::min<long long>(rows, cols);
    double* U = ar.alloc<double>((size_t)rows * kk);
    double* S = ar.alloc<double>(kk);
    std::vector<double> sv(kk);
    double* Vt = nullptr;   // tall case: the right factor
    if (cols > rows) {
      double* G = ar.alloc<double>((size_t)rows * rows);
      gemm<double>(s, false, true, rows, rows, (int)cols, 1.0, C, rows, 0, C, rows, 0, 0.0, G, rows, 0);
      double* Vg = ar.alloc<double>((size_t)rows * rows);
      svd<double>(s, ar, rows, rows, G, rows, U, rows, S, Vg, rows);
      QTT_CUDA(cudaMemcpyAsync(sv.data(), S, sizeof(double) * kk, cudaMemcpyDeviceToHost, s));
      QTT_CUDA(cudaStreamSynchronize(s));
      for (double& x : sv) x = std::sqrt(std::max(0.0, x));
    } else {
      double* A = ar.alloc<double>((size_t)rows * cols);
      QTT_CUDA(cudaMemcpyAsync(A, C, sizeof(double) * rows * cols, cudaMemcpyDeviceToDevice, s));
      Vt = ar.alloc<double>((size_t)kk * cols);
      svd<double>(s, ar, rows, (int)cols, A, rows, U, rows, S, Vt, kk);
      QTT_CUDA(cudaMemcpyAsync(sv.data(), S, sizeof(double) * kk, cudaMemcpyDeviceToHost, s));
      QTT_CUDA(cudaStreamSynchronize(s));
    }
    if (delta < 0.0) {
      double nrm2 = 0.0;
      for (double x : sv) nrm2 += x * x;
      delta = eps * std::sqrt(nrm2) / std::sqrt((double)std::max(1, d - 1));
    }
    const int rk = std::max(1, truncation_rank(sv, delta, max_rank, nullptr));
    double* Uk = ar.alloc<double>((size_t)rows * rk);
    copy2d<double>(s, rows, rk, U, rows, Uk, rows);
    core[k] = Uk;
    double* Cn = ar.alloc<double>((size_t)rk * cols);
    if (Vt) {
      // C_{k+1} = diag(S_k) Vt_k (leading rk rows)
      scale_rows_kernel<<<grid_for((long long)rk * cols), 256, 0, s>>>(rk, cols, Vt, kk, S, Cn);
      QTT_CHECK_LAUNCH();
    } else {
      // C_{k+1} = U_k^T C_k, in column blocks that keep the GEMM grid's
      // second dimension within its limit
      constexpr long long kBlock = 1LL << 20;
      for (long long c0 = 0; c0 < cols; c0 += kBlock) {
        const int nc = (int)std::min(kBlock, cols - c0);
        gemm<double>(s, true, false, rk, nc, rows, 1.0, Uk, rows, 0, C + c0 * rows, rows, 0, 0.0, Cn + c0 * rk, rk,
                     0);
      }
    }
    C = Cn;
    rprev = rk;
    r[k + 1] = rk;
  }
  core[d - 1] = C;
  qtt_tensor* t = tensor_alloc(d, n, ones.data(), r.data(), QTT_F64, 0);
  for (int k = 0; k < d; ++k)
    QTT_CUDA(cudaMemcpyAsync(t->core[k], core[k], sizeof(double) * (size_t)r[k] * n[k] * r[k + 1],
                             cudaMemcpyDeviceToDevice, s));
  return t;
}

namespace {
template <typename T>
__global__ void scale_columns_kernel(int rows, int cols, const T* __restrict__ A, int lda, const T* __restrict__ S,
                                     T* __restrict__ B, int ldb) {
  long long total = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % rows), j = (int)(t / rows);
    B[i + (long long)j * ldb] = A[i + (long long)j * lda] * S[j];
  }
}
}  // namespace

template <typename T>
void scale_columns(cudaStream_t s, int rows, int cols, const T* A, int lda, const T* S, T* B, int ldb) {
  if (rows <= 0 || cols <= 0) return;
  scale_columns_kernel<T><<<grid_for((long long)rows * cols), 256, 0, s>>>(rows, cols, A, lda, S, B, ldb);
  QTT_CHECK_LAUNCH();
}

#define QTT_INST_TT(T)                                                                                           \
  template void core_product<T>(cudaStream_t, int, int, int, int, int, int, int, const T*, const T*, T*);        \
  template void to_full<T>(cudaStream_t, Arena&, const qtt_tensor*, T*, size_t, int);                            \
  template qtt_tensor* product<T>(cudaStream_t, const qtt_tensor*, const qtt_tensor*);                           \
  template qtt_tensor* tt_sum<T>(cudaStream_t, T, const qtt_tensor*, T, const qtt_tensor*);                      \
  template void left_orthogonalize<T>(cudaStream_t, Arena&, qtt_tensor*, int);                                   \
  template void right_orthogonalize<T>(cudaStream_t, Arena&, qtt_tensor*, int);                                  \
  template double norm<T>(cudaStream_t, Arena&, const qtt_tensor*);                                              \
  template int round_tt<T>(cudaStream_t, Arena&, qtt_tensor*, double, int);                                      \
  template void scale_columns<T>(cudaStream_t, int, int, const T*, int, const T*, T*, int);                    \
  template void from_canonical<T>(cudaStream_t, const T*, T*, int, int);
QTT_INST_TT(double)
QTT_INST_TT(float)

}  // namespace qtt
