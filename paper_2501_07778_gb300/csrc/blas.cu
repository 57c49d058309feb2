// Dense building blocks: tiled GEMM, N-d permutation, reductions, and a
// two-operand Einstein-summation planner that maps every TT contraction of
// the engine onto (permute, strided-batched GEMM, permute).
#include <algorithm>
#include <cstring>
#include <string>

#include "common.cuh"
#include "contract.cuh"

namespace qtt {

// ---------------------------------------------------------------------------
// GEMM: TS x TS output tile per 256-thread block (TS = 64, or 32 when 64 x 64
// tiles cannot fill the SMs), 16-deep K slices staged in shared memory,
// (TS/16) x (TS/16) register tile per thread (rows tx + 16 i, cols ty + 16 j
// so that shared-memory reads are conflict-free).
// ---------------------------------------------------------------------------
namespace {
constexpr int GBM = 64, GBK = 16;

// gridDim.z = batch * splits: a split computes the partial product over
// K range [split * kchunk, min(K, (split + 1) * kchunk)) and, when splits > 1,
// adds alpha * partial into C atomically (C pre-scaled by beta on the host side).
template <typename T, int TS>
__global__ void __launch_bounds__(256) gemm_kernel(bool tA, bool tB, int M, int N, int K, T alpha, const T* __restrict__ A,
                                                  int lda, long long sA, const T* __restrict__ B, int ldb,
                                                  long long sB, T beta, T* __restrict__ C, int ldc, long long sC,
                                                  int splits, int kchunk) {
  constexpr int R = TS / 16, LOADS = GBK * TS / 256;
  __shared__ T As[GBK][TS + 1];
  __shared__ T Bs[GBK][TS + 1];
  const int bz = blockIdx.z / splits, sp = blockIdx.z % splits;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int kb = sp * kchunk, ke = min(K, kb + kchunk);
  const int m0 = blockIdx.x * TS, n0 = blockIdx.y * TS;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = T(0);
  for (int k0 = kb; k0 < ke; k0 += GBK) {
#pragma unroll
    for (int t = 0; t < LOADS; ++t) {
      int L = tid + 256 * t;
      int i, k;
      if (!tA) { i = L % TS; k = L / TS; } else { k = L % GBK; i = L / GBK; }
      int gi = m0 + i, gk = k0 + k;
      T v = T(0);
      if (gi < M && gk < ke) v = tA ? A[gk + (long long)gi * lda] : A[gi + (long long)gk * lda];
      As[k][i] = v;
      int j, kk;
      if (!tB) { kk = L % GBK; j = L / GBK; } else { j = L % TS; kk = L / TS; }
      int gj = n0 + j, gk2 = k0 + kk;
      T w = T(0);
      if (gj < N && gk2 < ke) w = tB ? B[gj + (long long)gk2 * ldb] : B[gk2 + (long long)gj * ldb];
      Bs[kk][j] = w;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GBK; ++k) {
      T a[R], b[R];
#pragma unroll
      for (int i = 0; i < R; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) b[j] = Bs[k][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int gi = m0 + tx + 16 * i;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      int gj = n0 + ty + 16 * j;
      if (gj >= N) continue;
      T* c = C + gi + (long long)gj * ldc;
      if (splits > 1) atomicAdd(c, alpha * acc[i][j]);
      else *c = (beta == T(0)) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*c);
    }
  }
}

template <typename T>
__global__ void scale_matrix_kernel(int M, int N, T* C, int ldc, long long sC, int batch, T beta) {
  long long total = (long long)M * N * batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % M);
    long long r = t / M;
    int j = (int)(r % N), b = (int)(r / N);
    T* c = C + b * sC + i + (long long)j * ldc;
    *c = (beta == T(0)) ? T(0) : beta * (*c);
  }
}

// Small-K / skinny fallback is not needed: the tile kernel handles any shape.

// Work-item loop over the strided contraction (contract.cuh): one block per
// TS x TS output tile (and K split), grid-strided.
template <typename T, int TS>
__global__ void __launch_bounds__(256) contract_kernel(ContractArgs a, T alpha, const T* __restrict__ A,
                                                       const T* __restrict__ B, T beta, T* __restrict__ C,
                                                       long long items) {
  __shared__ ContractSmem<T, TS> sm;
  for (long long it = blockIdx.x; it < items; it += gridDim.x)
    contract_tile<T, TS>(a, alpha, A, B, beta, C, (int)it, sm);
}

// C = beta C over the strided output (before split-K accumulation)
template <typename T>
__global__ void contract_scale_kernel(ContractArgs a, T* C, T beta) {
  long long total = (long long)a.M * a.N * a.batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    T* c = C + contract_out_off(a, t);
    *c = (beta == T(0)) ? T(0) : beta * (*c);
  }
}

constexpr int PMAX = 24;
struct PermArgs {
  int nd;
  long long out_dims[PMAX];
  long long in_stride[PMAX];   // input stride of output dim k
};

template <typename T>
__global__ void permute_kernel(const T* __restrict__ in, T* __restrict__ out, long long total, PermArgs a, T alpha,
                               T beta) {
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
       o += (long long)gridDim.x * blockDim.x) {
    long long rem = o, off = 0;
    for (int k = 0; k < a.nd; ++k) {
      long long c = rem % a.out_dims[k];
      rem /= a.out_dims[k];
      off += c * a.in_stride[k];
    }
    T v = alpha * in[off];
    out[o] = (beta == T(0)) ? v : v + beta * out[o];
  }
}

template <typename T>
__global__ void fill_kernel(T* p, size_t n, T v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

template <typename T>
__global__ void axpby_kernel(size_t n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (b == T(0)) ? a * x[i] : a * x[i] + b * y[i];
}

template <typename T>
__global__ void copy2d_kernel(int rows, int cols, const T* __restrict__ src, int lds, T* __restrict__ dst, int ldd) {
  long long total = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % rows);
    long long j = t / rows;
    dst[i + j * ldd] = src[i + j * lds];
  }
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void dot_kernel(const T* __restrict__ x, const T* __restrict__ y, size_t n, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc += (double)x[i] * (double)(y ? y[i] : x[i]);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) atomicAdd(out, v);
  }
}

inline int grid_for(long long n, int block = 256) { return grid_for_n(n, 16, block); }
}  // namespace

template <typename T>
void gemm(cudaStream_t s, bool tA, bool tB, int M, int N, int K, T alpha, const T* A, int lda, long long sA,
          const T* B, int ldb, long long sB, T beta, T* C, int ldc, long long sC, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    // C = beta C
    for (int b = 0; b < batch; ++b) {
      if (beta == T(0)) {
        for (int j = 0; j < N; ++j) QTT_CUDA(cudaMemsetAsync(C + b * sC + (long long)j * ldc, 0, sizeof(T) * M, s));
      } else {
        // rare; handled by scaling column-wise via axpby on contiguous runs
        for (int j = 0; j < N; ++j) axpby<T>(s, M, T(0), C + b * sC + (long long)j * ldc, beta, C + b * sC + (long long)j * ldc);
      }
    }
    return;
  }
  // FP64 runs at about 7 GFLOP/s per SM on this GPU: a GEMM whose 64 x 64
  // tiles leave SMs idle takes 32 x 32 tiles, and is split down to 32-deep K
  // chunks when even those cannot fill the SMs twice over
  const long long two_waves = 2LL * num_sms();
  auto tiles_of = [&](int ts) { return (long long)((M + ts - 1) / ts) * ((N + ts - 1) / ts) * batch; };
  const int TS = (sizeof(T) == 8 && tiles_of(GBM) < two_waves) ? 32 : GBM;
  const long long tiles = tiles_of(TS);
  int splits = 1;
  if (tiles < two_waves && K >= 64) {
    long long want = (two_waves + tiles - 1) / tiles;
    splits = (int)std::min<long long>(want, (K + 31) / 32);
    splits = std::max(1, std::min(splits, 65535 / std::max(1, batch)));
  }
  int kchunk = K;
  if (splits > 1) {
    kchunk = ((K + splits - 1) / splits + GBK - 1) / GBK * GBK;
    splits = (K + kchunk - 1) / kchunk;
  }
  dim3 grid((M + TS - 1) / TS, (N + TS - 1) / TS, batch * splits);
  QTT_REQUIRE(grid.y <= 65535 && grid.z <= 65535, "gemm grid too large");
  ProfToken pt = prof_begin(sizeof(T) == 8 ? PROF_GEMM_F64 : PROF_GEMM_F32, s);
  if (splits > 1) {
    long long total = (long long)M * N * batch;
    scale_matrix_kernel<T><<<grid_for(total), 256, 0, s>>>(M, N, C, ldc, sC, batch, beta);
    QTT_CHECK_LAUNCH();
  }
  if (TS == 32)
    gemm_kernel<T, 32><<<grid, 256, 0, s>>>(tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, splits,
                                            kchunk);
  else
    gemm_kernel<T, GBM><<<grid, 256, 0, s>>>(tA, tB, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC,
                                             splits, kchunk);
  QTT_CHECK_LAUNCH();
  if (pt.ev) {
    const double mn = (double)M * N, b = (double)batch;
    prof_end(pt, s, 2.0 * mn * K * b,
             b * sizeof(T) * ((double)M * K + (double)K * N + (beta == T(0) ? 1.0 : 2.0) * mn));
  }
}

template <typename T>
void permute(cudaStream_t s, const T* in, T* out, int nd, const int* dims, const int* perm, T alpha, T beta) {
  QTT_REQUIRE(nd >= 1 && nd <= PMAX, "permute: too many dimensions");
  long long stride[PMAX];
  long long acc = 1, total = 1;
  for (int k = 0; k < nd; ++k) {
    stride[k] = acc;
    acc *= dims[k];
  }
  PermArgs a;
  a.nd = nd;
  for (int k = 0; k < nd; ++k) {
    a.out_dims[k] = dims[perm[k]];
    a.in_stride[k] = stride[perm[k]];
    total *= dims[k];
  }
  if (total == 0) return;
  ProfToken pt = prof_begin(PROF_PERMUTE, s);
  permute_kernel<T><<<grid_for(total), 256, 0, s>>>(in, out, total, a, alpha, beta);
  QTT_CHECK_LAUNCH();
  if (pt.ev) prof_end(pt, s, 0.0, (double)total * sizeof(T) * (beta == T(0) ? 2.0 : 3.0));
}

template <typename T>
void fill(cudaStream_t s, T* p, size_t n, T v) {
  if (n == 0) return;
  fill_kernel<T><<<grid_for((long long)n), 256, 0, s>>>(p, n, v);
  QTT_CHECK_LAUNCH();
}

template <typename T>
void axpby(cudaStream_t s, size_t n, T a, const T* x, T b, T* y) {
  if (n == 0) return;
  axpby_kernel<T><<<grid_for((long long)n), 256, 0, s>>>(n, a, x, b, y);
  QTT_CHECK_LAUNCH();
}

template <typename T>
void copy2d(cudaStream_t s, int rows, int cols, const T* src, int lds, T* dst, int ldd) {
  if (rows <= 0 || cols <= 0) return;
  copy2d_kernel<T><<<grid_for((long long)rows * cols), 256, 0, s>>>(rows, cols, src, lds, dst, ldd);
  QTT_CHECK_LAUNCH();
}

template <typename S, typename D>
void convert(cudaStream_t s, const S* src, D* dst, size_t n) {
  if (n == 0) return;
  convert_kernel<S, D><<<grid_for((long long)n), 256, 0, s>>>(src, dst, n);
  QTT_CHECK_LAUNCH();
}

template <typename T>
void sumsq(cudaStream_t s, const T* x, size_t n, double* out) {
  QTT_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  if (n == 0) return;
  dot_kernel<T><<<std::min(grid_for((long long)n), 2 * num_sms()), 256, 0, s>>>(x, (const T*)nullptr, n, out);
  QTT_CHECK_LAUNCH();
}

template <typename T>
void dotp(cudaStream_t s, const T* x, const T* y, size_t n, double* out) {
  QTT_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  if (n == 0) return;
  dot_kernel<T><<<std::min(grid_for((long long)n), 2 * num_sms()), 256, 0, s>>>(x, y, n, out);
  QTT_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// Einsum planner.
// ---------------------------------------------------------------------------
namespace {
struct Operand {
  std::string lab;
  std::vector<int> dim;
};

std::string concat(const std::string& a, const std::string& b, const std::string& c) { return a + b + c; }

// permutation vector taking `have` layout to `want` layout (out dim k = in dim perm[k])
std::vector<int> perm_of(const std::string& have, const std::string& want) {
  std::vector<int> p(want.size());
  for (size_t k = 0; k < want.size(); ++k) p[k] = (int)have.find(want[k]);
  return p;
}

long long prod_of(const std::string& labs, const int* size_of) {
  long long p = 1;
  for (char c : labs) p *= size_of[(unsigned char)c];
  return p;
}

// labels of `group` in the order they appear in `order`
std::string ordered(const std::string& group, const std::string& order) {
  std::string out;
  for (char c : order)
    if (group.find(c) != std::string::npos) out += c;
  return out;
}
}  // namespace

template <typename T>
void einsum(cudaStream_t s, Arena& ar, const char* spec, const T* A, const int* dA, const T* B, const int* dB, T* C,
            T alpha, T beta) {
  std::string sp(spec);
  size_t comma = sp.find(','), arrow = sp.find("->");
  QTT_REQUIRE(comma != std::string::npos && arrow != std::string::npos, "einsum: bad spec");
  std::string la = sp.substr(0, comma), lb = sp.substr(comma + 1, arrow - comma - 1), lc = sp.substr(arrow + 2);
  int size_of[256];
  for (int i = 0; i < 256; ++i) size_of[i] = -1;
  for (size_t k = 0; k < la.size(); ++k) size_of[(unsigned char)la[k]] = dA[k];
  for (size_t k = 0; k < lb.size(); ++k) {
    int& z = size_of[(unsigned char)lb[k]];
    QTT_REQUIRE(z < 0 || z == dB[k], std::string("einsum: size mismatch for label ") + lb[k] + " in " + sp);
    z = dB[k];
  }
  std::string batch, contr, freeA, freeB;
  for (char c : la) {
    bool inB = lb.find(c) != std::string::npos, inC = lc.find(c) != std::string::npos;
    if (inB && inC) batch += c;
    else if (inB) contr += c;
    else if (inC) freeA += c;
    else QTT_REQUIRE(false, "einsum: label only in A");
  }
  for (char c : lb) {
    bool inA = la.find(c) != std::string::npos, inC = lc.find(c) != std::string::npos;
    if (!inA) {
      QTT_REQUIRE(inC, "einsum: label only in B");
      freeB += c;
    }
  }
  for (char c : lc) QTT_REQUIRE(size_of[(unsigned char)c] >= 0, "einsum: output label not in inputs");
  // within-group orders: free groups follow the output, batch follows the output
  batch = ordered(batch, lc);
  freeA = ordered(freeA, lc);
  freeB = ordered(freeB, lc);
  // contracted order: from A if that lets A stay unpermuted, else from B
  std::string cA = ordered(contr, la), cB = ordered(contr, lb);
  auto a_ok = [&](const std::string& c) {
    return la == concat(freeA, c, batch) || la == concat(c, freeA, batch);
  };
  contr = a_ok(cA) ? cA : cB;
  const long long nFA = prod_of(freeA, size_of), nFB = prod_of(freeB, size_of), nK = prod_of(contr, size_of),
                  nBt = prod_of(batch, size_of);
  QTT_REQUIRE(nBt <= 65535, "einsum: batch too large");
  if (nFA == 0 || nFB == 0 || nBt == 0) return;
  {
    ContractArgs ca{};
    if (plan_contract(spec, dA, dB, (int)sizeof(T), 2LL * num_sms(), ca, sizeof(T) == 8)) {
      const long long items = contract_items(ca);
      ProfToken pt = prof_begin(sizeof(T) == 8 ? PROF_GEMM_F64 : PROF_GEMM_F32, s);
      if (ca.splits > 1) {
        contract_scale_kernel<T><<<grid_for((long long)ca.M * ca.N * ca.batch), 256, 0, s>>>(ca, C, beta);
        QTT_CHECK_LAUNCH();
      }
      const int grid = (int)std::min<long long>(items, 1LL << 30);
      if (ca.tile == 32) contract_kernel<T, 32><<<grid, 256, 0, s>>>(ca, alpha, A, B, beta, C, items);
      else contract_kernel<T, CT_BM><<<grid, 256, 0, s>>>(ca, alpha, A, B, beta, C, items);
      QTT_CHECK_LAUNCH();
      if (pt.ev) {
        const double mn = (double)ca.M * ca.N, bt = (double)ca.batch;
        prof_end(pt, s, 2.0 * mn * ca.K * bt,
                 bt * sizeof(T) * ((double)ca.M * ca.K + (double)ca.K * ca.N + (beta == T(0) ? 1.0 : 2.0) * mn));
      }
      return;
    }
  }
  // operand A
  const T* Ause = A;
  bool tA = false;
  if (la == concat(freeA, contr, batch)) {
    tA = false;
  } else if (la == concat(contr, freeA, batch)) {
    tA = true;
  } else {
    std::string want = concat(freeA, contr, batch);
    std::vector<int> p = perm_of(la, want);
    T* tmp = ar.alloc<T>(nFA * nK * nBt);
    permute<T>(s, A, tmp, (int)la.size(), dA, p.data());
    Ause = tmp;
    tA = false;
  }
  const T* Buse = B;
  bool tB = false;
  if (lb == concat(contr, freeB, batch)) {
    tB = false;
  } else if (lb == concat(freeB, contr, batch)) {
    tB = true;
  } else {
    std::string want = concat(contr, freeB, batch);
    std::vector<int> p = perm_of(lb, want);
    T* tmp = ar.alloc<T>(nK * nFB * nBt);
    permute<T>(s, B, tmp, (int)lb.size(), dB, p.data());
    Buse = tmp;
    tB = false;
  }
  const int lda = tA ? (int)nK : (int)nFA;
  const int ldb = tB ? (int)nFB : (int)nK;
  const long long sA = nFA * nK, sB = nK * nFB, sCs = nFA * nFB;
  if (lc == concat(freeA, freeB, batch)) {
    gemm<T>(s, tA, tB, (int)nFA, (int)nFB, (int)nK, alpha, Ause, lda, sA, Buse, ldb, sB, beta, C, (int)nFA, sCs,
            (int)nBt);
  } else if (lc == concat(freeB, freeA, batch)) {
    // C^T = op(B)^T op(A)^T
    gemm<T>(s, !tB, !tA, (int)nFB, (int)nFA, (int)nK, alpha, Buse, ldb, sB, Ause, lda, sA, beta, C, (int)nFB, sCs,
            (int)nBt);
  } else {
    T* tmp = ar.alloc<T>(nFA * nFB * nBt);
    gemm<T>(s, tA, tB, (int)nFA, (int)nFB, (int)nK, T(1), Ause, lda, sA, Buse, ldb, sB, T(0), tmp, (int)nFA, sCs,
            (int)nBt);
    std::string have = concat(freeA, freeB, batch);
    std::vector<int> dims(have.size());
    for (size_t k = 0; k < have.size(); ++k) dims[k] = size_of[(unsigned char)have[k]];
    std::vector<int> p = perm_of(have, lc);
    permute<T>(s, tmp, C, (int)have.size(), dims.data(), p.data(), alpha, beta);
  }
}


// ---------------------------------------------------------------------------
// Contraction planner (contract.cuh)
// ---------------------------------------------------------------------------
bool plan_contract(const char* spec, const int* dA, const int* dB, int sizeof_T, long long min_items,
                   ContractArgs& ca, bool allow_small) {
  std::string sp(spec);
  size_t comma = sp.find(','), arrow = sp.find("->");
  QTT_REQUIRE(comma != std::string::npos && arrow != std::string::npos, "contract: bad spec");
  std::string la = sp.substr(0, comma), lb = sp.substr(comma + 1, arrow - comma - 1), lc = sp.substr(arrow + 2);
  int size_of[256];
  for (int i = 0; i < 256; ++i) size_of[i] = -1;
  for (size_t k = 0; k < la.size(); ++k) size_of[(unsigned char)la[k]] = dA[k];
  for (size_t k = 0; k < lb.size(); ++k) {
    int& z = size_of[(unsigned char)lb[k]];
    QTT_REQUIRE(z < 0 || z == dB[k], std::string("contract: size mismatch for label ") + lb[k] + " in " + sp);
    z = dB[k];
  }
  std::string batch, contr, freeA, freeB;
  for (char c : la) {
    bool inB = lb.find(c) != std::string::npos, inC = lc.find(c) != std::string::npos;
    if (inB && inC) batch += c;
    else if (inB) contr += c;
    else if (inC) freeA += c;
    else QTT_REQUIRE(false, "contract: label only in A");
  }
  for (char c : lb)
    if (la.find(c) == std::string::npos) {
      QTT_REQUIRE(lc.find(c) != std::string::npos, "contract: label only in B");
      freeB += c;
    }
  if (freeA.size() > 4 || freeB.size() > 4 || contr.size() > 4 || batch.size() > 4) return false;
  auto prod = [&](const std::string& g) {
    long long p = 1;
    for (char c : g) p *= size_of[(unsigned char)c];
    return p;
  };
  const long long nFA = prod(freeA), nFB = prod(freeB), nK = prod(contr), nBt = prod(batch);
  if (nFA >= (1LL << 31) || nFB >= (1LL << 31) || nK >= (1LL << 31) || nBt > 65535) return false;
  auto strides = [&](const std::string& lab) {
    std::vector<long long> st(256, 0);
    long long acc = 1;
    for (char c : lab) {
      st[(unsigned char)c] = acc;
      acc *= size_of[(unsigned char)c];
    }
    return st;
  };
  std::vector<long long> sa = strides(la), sb = strides(lb), sc = strides(lc);
  auto sort_by = [&](std::string g, const std::vector<long long>& st) {
    std::stable_sort(g.begin(), g.end(), [&](char x, char y) { return st[(unsigned char)x] < st[(unsigned char)y]; });
    return g;
  };
  const std::string gA = sort_by(freeA, sa), gB = sort_by(freeB, sb), gK = sort_by(contr, sa);
  auto make = [&](const std::string& g, const std::vector<long long>& st) {
    IdxMap m{};
    m.cnt = (int)g.size();
    for (int t = 0; t < m.cnt; ++t) {
      m.n[t] = size_of[(unsigned char)g[t]];
      m.s[t] = st[(unsigned char)g[t]];
    }
    if (m.cnt == 0) {
      m.cnt = 1;
      m.n[0] = 1;
      m.s[0] = 0;
    }
    return m;
  };
  ca = ContractArgs{};
  ca.M = (int)nFA;
  ca.N = (int)nFB;
  ca.K = (int)nK;
  ca.batch = (int)nBt;
  ca.am = make(gA, sa);
  ca.cm = make(gA, sc);
  ca.bn = make(gB, sb);
  ca.cn = make(gB, sc);
  ca.ak = make(gK, sa);
  ca.bk = make(gK, sb);
  ca.ab = make(batch, sa);
  ca.bb = make(batch, sb);
  ca.cb = make(batch, sc);
  ca.a_m_fast = (ca.am.s[0] == 1) || !(ca.ak.s[0] == 1);
  ca.b_n_fast = (ca.bn.s[0] == 1) && !(ca.bk.s[0] == 1);
  auto tiles_of = [&](int ts) { return ((nFA + ts - 1) / ts) * ((nFB + ts - 1) / ts) * nBt; };
  ca.tile = (allow_small && tiles_of(CT_BM) < min_items) ? 32 : CT_BM;
  ca.tiles_m = (int)((nFA + ca.tile - 1) / ca.tile);
  ca.tiles_n = (int)((nFB + ca.tile - 1) / ca.tile);
  const long long tiles = tiles_of(ca.tile);
  int splits = 1;
  if (tiles < min_items && nK >= 64) {
    long long want = (min_items + tiles - 1) / tiles;
    splits = (int)std::min<long long>(want, (nK + 31) / 32);
    splits = std::max(1, splits);
  }
  int kchunk = (int)std::max<long long>(1, nK);
  if (splits > 1) {
    kchunk = (int)(((nK + splits - 1) / splits + CT_BK - 1) / CT_BK * CT_BK);
    splits = (int)((nK + kchunk - 1) / kchunk);
  }
  ca.splits = splits;
  ca.kchunk = kchunk;
  (void)sizeof_T;
  return true;
}

#define QTT_INST(T)                                                                                              \
  template void gemm<T>(cudaStream_t, bool, bool, int, int, int, T, const T*, int, long long, const T*, int,    \
                        long long, T, T*, int, long long, int);                                                  \
  template void permute<T>(cudaStream_t, const T*, T*, int, const int*, const int*, T, T);                       \
  template void fill<T>(cudaStream_t, T*, size_t, T);                                                            \
  template void axpby<T>(cudaStream_t, size_t, T, const T*, T, T*);                                              \
  template void copy2d<T>(cudaStream_t, int, int, const T*, int, T*, int);                                       \
  template void sumsq<T>(cudaStream_t, const T*, size_t, double*);                                               \
  template void dotp<T>(cudaStream_t, const T*, const T*, size_t, double*);                                      \
  template void einsum<T>(cudaStream_t, Arena&, const char*, const T*, const int*, const T*, const int*, T*, T, T);
QTT_INST(double)
QTT_INST(float)
template void convert<double, float>(cudaStream_t, const double*, float*, size_t);
template void convert<float, double>(cudaStream_t, const float*, double*, size_t);
template void convert<double, double>(cudaStream_t, const double*, double*, size_t);
template void convert<float, float>(cudaStream_t, const float*, float*, size_t);

}  // namespace qtt
