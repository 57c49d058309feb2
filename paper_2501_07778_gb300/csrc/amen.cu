// qtt_solve: one-site AMEn with residual-based enrichment (Dolgov &
// Savostyanov 2014, the solver the paper uses for K u = f), restated for
// this engine:
//   right-orthogonalise x and the residual proxy z; build right interfaces
//   Phi_R(x,K,x), Psi_R(x,f), Phi_R(z,K,x), Psi_R(z,f);
//   for k = 1..D: local Galerkin system B_k = Phi_L K_k Phi_R, local rhs g_k;
//     record ||B_k x_k - g_k|| / ||g_k||; solve (dense LU, Jacobi-
//     preconditioned CG for a symmetric K, restarted GMRES otherwise);
//     truncate the left unfolding by SVD at the smallest rank whose local
//     residual stays within tol / sqrt(D); new z core = orth of the
//     residual projected on z's interfaces; enrich [U, residual projected on
//     x's left and z's right interfaces], orthogonalise, push the remainder
//     into core k+1; update the left interfaces;
//   stop when the sweep's largest local residual is <= tol, or (FP64
//   interfaces) when the FP64 global residual is <= tol.
// QTT_F64 and QTT_MIXED keep interfaces and residuals in FP64; QTT_MIXED
// runs the local Krylov iterations on an FP32 copy of the local operator.
// When the sweeps stall above tol, both refine: r = f - K u rounded in FP64
// by randomized TT rounding (residual.cu), K d = r solved the same way to a
// looser tolerance, u <- u + d.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>

#include "common.cuh"
#include "contract.cuh"
#include "tc_gemm.cuh"
#include "tt_ops.cuh"

namespace qtt {
double residual64(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f);
bool has_fe_operator(const qtt_tensor* K);
qtt_tensor* residual_fe_tt(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f, double eps,
                           int max_rank, double* rel);
// The refinement forms its residual element by element (TT-SVD, ranks
// <= kFeResidualRank) once the FP64 relative residual is below
// kFeResidualBelow, or once a correction from the QTT-formed residual has
// failed to halve the residual.  Measured: on the L = 10 plate at 5e-10 the residual
// formed in QTT arithmetic kept 4 % of K^-1 r, the element-by-element one
// (rank 128) kept it all and six refinements took the error against sparse
// direct from 5.2e-9 to 7e-10; on the L = 12 plates at 2-7e-8 the QTT
// residual reaches 1e-8 in one refinement, while the TT-SVD one is a second
// slower at rank 128 (FP64 Jacobi SVDs of 512 x 512 Gram matrices) and
// stalls above 1e-8 at rank 32.
constexpr int kFeResidualRank = 128;
constexpr double kFeResidualBelow = 1e-9;
double residual_fe(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* u2,
                   const qtt_tensor* f);
namespace {

// The FP64 global relative residual ||f - K (u + u2)|| / ||f|| (u2 may be
// NULL): for an MPO from qtt_assemble_stiffness, K is applied in full format
// as the finite-element operator it represents (fe_residual.cu, HBM-bound);
// otherwise by the exact QTT product, expanded (residual64).  Its count and
// host wall time go to the solve record.
double timed_residual64(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f,
                        qtt_solve_info* info, const qtt_tensor* u2 = nullptr) {
  const auto t0 = std::chrono::steady_clock::now();
  double rel;
  if (has_fe_operator(K)) {
    rel = residual_fe(s, K, u, u2, f);
  } else if (u2) {
    auto sum = tt_sum<double>(s, 1.0, u, 1.0, u2);
    try {
      rel = residual64(s, K, sum, f);
    } catch (...) {
      tensor_free(sum);
      throw;
    }
    tensor_free(sum);
  } else {
    rel = residual64(s, K, u, f);
  }
  if (info) {
    info->checks += 1;
    info->check_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return rel;
}

using Tptr = std::unique_ptr<qtt_tensor, void (*)(qtt_tensor*)>;
Tptr own(qtt_tensor* t) { return Tptr(t, tensor_free); }

inline int grid_for(long long n) { return grid_for_n(n, 32); }

// growable device buffer
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t cap = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), cap(o.cap), s(o.s) {
    o.p = nullptr;
    o.cap = 0;
  }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      if (p) cudaFreeAsync(p, s);
      p = o.p;
      cap = o.cap;
      s = o.s;
      o.p = nullptr;
      o.cap = 0;
    }
    return *this;
  }
  void swap(DBuf& o) noexcept {
    std::swap(p, o.p);
    std::swap(cap, o.cap);
    std::swap(s, o.s);
  }
  void ensure(size_t n, cudaStream_t st) {
    s = st;
    if (n <= cap) return;
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    size_t c = std::max<size_t>(n, cap * 3 / 2);
    count_alloc();
    cudaError_t e = cudaMallocAsync(&p, c * sizeof(T), s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw QttError(QTT_ENOMEM, "solver buffer allocation failed");
    }
    cap = c;
  }
  ~DBuf() {
    if (p) cudaFreeAsync(p, s);
  }
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
template <typename T>
__global__ void scale_by_device_kernel(T* v, const T* src, int n, const double* nrm2, double* hout) {
  double h = sqrt(*nrm2);
  if (blockIdx.x == 0 && threadIdx.x == 0 && hout) *hout = h;
  double inv = h > 0 ? 1.0 / h : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = (T)((double)src[i] * inv);
}

// out += sum_i (a_i - b_i)^2 with a in FP32 and b in T, accumulated in FP64
template <typename T>
__global__ void diff_sumsq_kernel(const float* __restrict__ a, const T* __restrict__ b, int n, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double d = (double)a[i] - (double)b[i];
    acc += d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(out, v);
  }
}

// Givens least squares for min || beta e1 - H y ||, H (m+1) x m (ld m+1),
// single thread block; writes y (m) and the residual estimate
__global__ void gmres_lsq_kernel(const double* H, int m, double beta, double* y, double* res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double R[65 * 64];
  double g[65];
  const int ld = m + 1;
  for (int j = 0; j < m; ++j)
    for (int i = 0; i <= m; ++i) R[i + ld * j] = H[i + ld * j];
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  for (int j = 0; j < m; ++j) {
    double a = R[j + ld * j], b = R[j + 1 + ld * j];
    double r = sqrt(a * a + b * b);
    double c = r > 0 ? a / r : 1.0, s = r > 0 ? b / r : 0.0;
    for (int k = j; k < m; ++k) {
      double x1 = R[j + ld * k], x2 = R[j + 1 + ld * k];
      R[j + ld * k] = c * x1 + s * x2;
      R[j + 1 + ld * k] = -s * x1 + c * x2;
    }
    double g1 = g[j], g2 = g[j + 1];
    g[j] = c * g1 + s * g2;
    g[j + 1] = -s * g1 + c * g2;
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = g[i];
    for (int k = i + 1; k < m; ++k) v -= R[i + ld * k] * y[k];
    double d = R[i + ld * i];
    y[i] = d != 0.0 ? v / d : 0.0;
  }
  *res = fabs(g[m]);
}

template <typename T>
__global__ void store_col_kernel(double* H, int ldh, int j, const T* h, int len, const double* hlast) {
  int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i < len) H[i + (long long)ldh * j] = (double)h[i];
  if (i == 0 && hlast) H[len + (long long)ldh * j] = *hlast;
}

template <typename T>
__global__ void to_T_kernel(const double* src, T* dst, int n) {
  int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i < n) dst[i] = (T)src[i];
}

template <typename T>
__global__ void scale_rows_kernel(int rows, int cols, const T* A, int lda, const T* S, T* B, int ldb) {
  long long total = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % rows), j = (int)(t / rows);
    B[i + (long long)j * ldb] = A[i + (long long)j * lda] * S[i];
  }
}

// CG step with device scalars: alpha = rr / (p.Bp); d += alpha p; r -= alpha Bp
template <typename U>
__global__ void cg_step_kernel(U* d, U* r, const U* p, const U* q, const double* rr, const double* pq, int n) {
  const double den = *pq;
  const double alpha = den > 0.0 ? *rr / den : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    d[i] = (U)((double)d[i] + alpha * (double)p[i]);
    r[i] = (U)((double)r[i] - alpha * (double)q[i]);
  }
}

// Jacobi preconditioner of the local operator: the diagonal of
// Phi_L[a,A,a'] K[A,i,j,B] Phi_R[b,B,b'] at a = a', i = j, b = b' is
// sum_{A,B} Phi_L[a,A,a] K[A,i,i,B] Phi_R[b,B,b].
template <typename T>
__global__ void diag3_kernel(const T* P, int r, int R, T* out) {   // out[a + r X] = P[a + r (X + R a)]
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= r * R) return;
  int a = t % r, X = t / r;
  out[t] = P[a + (long long)r * (X + (long long)R * a)];
}

template <typename T>
__global__ void diagK_kernel(const T* K, int R0, int n, int R1, T* out) {   // out[A + R0 (i + n B)] = K[A,i,i,B]
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R0 * n * R1) return;
  int A = t % R0, i = (t / R0) % n, B = t / (R0 * n);
  out[t] = K[A + (long long)R0 * (i + (long long)n * (i + (long long)n * B))];
}

template <typename T, typename U>
__global__ void inv_diag_kernel(const T* diag, U* minv, int N) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const double v = (double)diag[t];
  minv[t] = (U)(v > 0.0 ? 1.0 / v : 1.0);
}

// z = m * r (elementwise)
template <typename U>
__global__ void precond_kernel(U* z, const U* m, const U* r, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) z[i] = m[i] * r[i];
}

// p = r + (rr_new / rr_old) p
template <typename U>
__global__ void cg_dir_kernel(U* p, const U* r, const double* rr_new, const double* rr_old, int n) {
  const double old = *rr_old;
  const double beta = old > 0.0 ? *rr_new / old : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = (U)((double)r[i] + beta * (double)p[i]);
}

// ---------------------------------------------------------------------------
// Persistent local CG (FP32): `iters` conjugate-gradient iterations on
// B d = r in one cooperative launch.  Per iteration: the three contractions
// of the local operator (p -> t1 -> t2 -> q) as grid-strided tile loops, the
// dot products as block reductions with atomic accumulation, the vector
// updates grid-strided; grid barriers separate the phases.  Device scalars:
// acc[0] = r.r of the current direction, acc[1] = p.Bp, acc[2] = new r.r.
// ---------------------------------------------------------------------------
struct PcgArgs {
  ContractArgs c1, c2, c3;
  const float* PL;
  const float* Ak;
  const float* PR;
  const float* minv;   // inverse diagonal of the local operator (Jacobi preconditioner)
  float* t1;
  float* t2;
  float* d;
  float* r;
  float* p;
  float* q;
  double* acc;
  int N, iters;
};

__device__ double block_reduce_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;   // valid in thread 0
}

__global__ void __launch_bounds__(256) pcg_kernel(PcgArgs a) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  __shared__ ContractSmem<float> sm;
  __shared__ double red[32];
  const long long it1 = contract_items(a.c1), it2 = contract_items(a.c2), it3 = contract_items(a.c3);
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gstride = (long long)gridDim.x * blockDim.x;
  for (int it = 0; it < a.iters; ++it) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && it > 0) {
      a.acc[0] = a.acc[2];
      a.acc[1] = 0.0;
      a.acc[2] = 0.0;
    }
    for (long long w = blockIdx.x; w < it1; w += gridDim.x) contract_tile<float>(a.c1, 1.f, a.p, a.PR, 0.f, a.t1, (int)w, sm);
    for (long long i = gtid; i < a.N; i += gstride) a.q[i] = 0.f;
    grid.sync();
    for (long long w = blockIdx.x; w < it2; w += gridDim.x) contract_tile<float>(a.c2, 1.f, a.t1, a.Ak, 0.f, a.t2, (int)w, sm);
    grid.sync();
    for (long long w = blockIdx.x; w < it3; w += gridDim.x) contract_tile<float>(a.c3, 1.f, a.PL, a.t2, 0.f, a.q, (int)w, sm);
    grid.sync();
    double part = 0.0;
    for (long long i = gtid; i < a.N; i += gstride) part += (double)a.p[i] * (double)a.q[i];
    part = block_reduce_sum(part, red);
    if (threadIdx.x == 0) atomicAdd(&a.acc[1], part);
    grid.sync();
    const double pq = a.acc[1];
    const double alpha = pq > 0.0 ? a.acc[0] / pq : 0.0;
    part = 0.0;
    for (long long i = gtid; i < a.N; i += gstride) {
      a.d[i] = (float)((double)a.d[i] + alpha * (double)a.p[i]);
      const float ri = (float)((double)a.r[i] - alpha * (double)a.q[i]);
      a.r[i] = ri;
      part += (double)ri * (double)ri * (double)a.minv[i];      // r . M^-1 r
    }
    part = block_reduce_sum(part, red);
    if (threadIdx.x == 0) atomicAdd(&a.acc[2], part);
    grid.sync();
    const double rr = a.acc[0];
    const double beta = rr > 0.0 ? a.acc[2] / rr : 0.0;
    for (long long i = gtid; i < a.N; i += gstride)
      a.p[i] = (float)((double)a.minv[i] * (double)a.r[i] + beta * (double)a.p[i]);
    grid.sync();
  }
}

// grid of the persistent CG: every SM holds up to two blocks (0 = the
// cooperative launch is unavailable; computed once per process).  A solve
// that shares the GPU with concurrent solves (batched workers) takes
// 1/g_gpu_share of it, so that the cooperative grids of different workers
// can be resident at the same time.
thread_local int g_gpu_share = 1;

int persistent_cg_grid_full() {
  static int grid = -1;
  if (grid >= 0) return grid;
  int dev = 0, coop = 0, sms = 0, nb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pcg_kernel, 256, 0) != cudaSuccess || !coop || nb < 1) {
    cudaGetLastError();
    grid = 0;
  } else {
    grid = sms * std::min(nb, 2);
  }
  return grid;
}

int persistent_cg_grid() {
  const int full = persistent_cg_grid_full();
  if (full <= 0) return 0;
  return std::max(8, full / std::max(1, g_gpu_share));
}

// deterministic residual proxy when none is given: smooth sign-varying values
template <typename T>
__global__ void proxy_kernel(T* c, long long n, int k) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c[i] = (T)sin(0.7 + 1.3 * (double)i + 2.1 * (double)k + 0.37 * (double)(i * i % 97));
}

// (B x)[a,i,b] = sum PhiL[a,A,c] K_k[A,i,j,B] PhiR[b,B,d] x[c,j,d], contracted
// over d, then (j, B), then (c, A); PhiL (ra,R0,rc), PhiR (rb,R1,rd), x (rc,n,rd)
template <typename U>
void apply_local(cudaStream_t s, Arena& sc, const U* PhiL, int ra, int rc, const U* Ak, int R0, int n, int R1,
                 const U* PhiR, int rb, int rd, const U* xk, U* out) {
  int dx[3] = {rc, n, rd}, dR[3] = {rb, R1, rd};
  U* t1 = sc.alloc<U>((size_t)rc * n * rb * R1);
  einsum<U>(s, sc, "cjd,bBd->cjbB", xk, dx, PhiR, dR, t1);
  int d1[4] = {rc, n, rb, R1}, dA[4] = {R0, n, n, R1};
  U* t2 = sc.alloc<U>((size_t)rc * rb * R0 * n);
  einsum<U>(s, sc, "cjbB,AijB->cbAi", t1, d1, Ak, dA, t2);
  int dL[3] = {ra, R0, rc}, d2[4] = {rc, rb, R0, n};
  einsum<U>(s, sc, "aAc,cbAi->aib", PhiL, dL, t2, d2, out);
}

// ---------------------------------------------------------------------------
// The FP32 local operator B p = Phi_L K_k Phi_R p on the tensor cores: the
// three contractions of apply_local as K-major 3xTF32 GEMMs (tc_gemm.cu),
//   t1[(c,b); (j,B)] = sum_d   p[(c,j); d]       Phi_R[(b,B); d]
//   t2[(i,b); (A,c)] = sum_jB  t1[(c,b); (j,B)]  K_k[(A,i); (j,B)]
//   q[a, i, b]       = sum_Ac  Phi_L[a; (A,c)]   t2[(i,b); (A,c)]
// where every epilogue writes its output directly in the K-major TF32-pair
// layout the next GEMM reads; the fixed factors are packed once per local
// solve, p once per application (the last GEMM splits its long K loop).
// ---------------------------------------------------------------------------
inline int pad4(int x) { return (x + 3) / 4 * 4; }

// ---------------------------------------------------------------------------
// Autotuner of the FP32 local operator.  Per GPU and per rank bucket of the
// local system (r0, r1 rounded down to half-octaves), the first local solve
// runs its Krylov iterations on the tensor cores (TcLocalOp), the next one
// in the persistent SIMT CG kernel; CUDA events give each one's time per
// iteration, and every later solve in the bucket takes the faster path.
// ---------------------------------------------------------------------------
struct TuneEntry {
  int dev, b0, b1;
  double us_tc = -1.0, us_simt = -1.0;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;

inline int half_octave(int r) { return (int)std::floor(2.0 * std::log2((double)std::max(1, r))); }

// 1: tensor cores, 0: SIMT, 2: time the tensor cores now, 3: time SIMT now
int tune_choice(int r0, int r1) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int b0 = half_octave(r0), b1 = half_octave(r1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& e : g_tune)
    if (e.dev == dev && e.b0 == b0 && e.b1 == b1) {
      if (e.us_tc < 0) return 2;
      if (e.us_simt < 0) return 3;
      return e.us_tc < e.us_simt ? 1 : 0;
    }
  g_tune.push_back(TuneEntry{dev, b0, b1});
  return 2;
}

void tune_record(int r0, int r1, bool tc, double us) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int b0 = half_octave(r0), b1 = half_octave(r1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& e : g_tune)
    if (e.dev == dev && e.b0 == b0 && e.b1 == b1) {
      if (tc && e.us_tc < 0) e.us_tc = us;
      if (!tc && e.us_simt < 0) e.us_simt = us;
      return;
    }
}

inline TcIdxMap idx1(int n0, long long s0) {
  TcIdxMap m{};
  m.cnt = 1;
  m.n[0] = n0;
  m.s[0] = s0;
  return m;
}
inline TcIdxMap idx2(int n0, long long s0, int n1, long long s1) {
  TcIdxMap m{};
  m.cnt = 2;
  m.n[0] = n0;
  m.s[0] = s0;
  m.n[1] = n1;
  m.s[1] = s1;
  return m;
}

struct TcLocalOp {
  int r0 = 0, n = 0, r1 = 0, R0 = 0, R1 = 0, ld1 = 0, ld2 = 0, ld3 = 0;
  float *pTh = nullptr, *pTl = nullptr;
  TcGemmPlan g1, g2, g3;

  // PL (r0, R0, r0), Ak (R0, n, n, R1), PR (r1, R1, r1): FP32, column-major;
  // q: the output vector (r0, n, r1)
  void build(cudaStream_t s, Arena& ar, const float* PL, const float* Ak, const float* PR, int r0_, int n_, int r1_,
             int R0_, int R1_, float* q) {
    r0 = r0_, n = n_, r1 = r1_, R0 = R0_, R1 = R1_;
    ld1 = pad4(r1);
    ld2 = pad4(n * R1);
    ld3 = pad4(R0 * r0);
    const int M1 = r0 * n, N1 = r1 * R1, M2 = r0 * r1, N2 = R0 * n, M3 = r0, N3 = n * r1;
    pTh = ar.alloc<float>((size_t)M1 * ld1);
    pTl = ar.alloc<float>((size_t)M1 * ld1);
    float* PRh = ar.alloc<float>((size_t)N1 * ld1);
    float* PRl = ar.alloc<float>((size_t)N1 * ld1);
    float* t1h = ar.alloc<float>((size_t)M2 * ld2);
    float* t1l = ar.alloc<float>((size_t)M2 * ld2);
    float* Kh = ar.alloc<float>((size_t)N2 * ld2);
    float* Kl = ar.alloc<float>((size_t)N2 * ld2);
    float* PLh = ar.alloc<float>((size_t)M3 * ld3);
    float* PLl = ar.alloc<float>((size_t)M3 * ld3);
    float* t2h = ar.alloc<float>((size_t)N3 * ld3);
    float* t2l = ar.alloc<float>((size_t)N3 * ld3);
    // fixed factors: Phi_R[(b,B); d], K[(A,i); (j,B)], Phi_L[a; (A,c)]
    tc_pack(s, PR, N1, r1, ld1, idx2(r1, 1, R1, r1), idx1(r1, (long long)r1 * R1), PRh, PRl);
    tc_pack(s, Ak, N2, n * R1, ld2, idx2(R0, 1, n, R0), idx2(n, (long long)R0 * n, R1, (long long)R0 * n * n), Kh, Kl);
    tc_pack(s, PL, M3, R0 * r0, ld3, idx1(r0, 1), idx2(R0, r0, r0, (long long)r0 * R0), PLh, PLl);
    TcEpilogue e1{};
    e1.om = idx2(r0, ld2, n, 1);                                   // (c, j) -> row c + r0 b, column j + n B
    e1.on = idx2(r1, (long long)r0 * ld2, R1, n);
    e1.out = t1h;
    e1.lo = t1l;
    tc_plan(g1, M1, N1, r1, pTh, pTl, ld1, PRh, PRl, ld1, e1, 1);
    TcEpilogue e2{};
    e2.om = idx2(r0, R0, r1, (long long)n * ld3);                  // (c, b) -> row i + n b, column A + R0 c
    e2.on = idx2(R0, 1, n, ld3);
    e2.out = t2h;
    e2.lo = t2l;
    tc_plan(g2, M2, N2, n * R1, t1h, t1l, ld2, Kh, Kl, ld2, e2, 1);
    TcEpilogue e3{};
    e3.om = idx1(r0, 1);                                           // q[a, i, b] at a + r0 (i + n b)
    e3.on = idx2(n, r0, r1, (long long)r0 * n);
    e3.out = q;
    e3.lo = nullptr;
    const long long tiles3 = (long long)((M3 + 127) / 128) * ((N3 + 127) / 128);
    const int want = (int)std::max<long long>(1, (2LL * num_sms() + tiles3 - 1) / tiles3);
    e3.atomic = want > 1 ? 1 : 0;
    tc_plan(g3, M3, N3, R0 * r0, PLh, PLl, ld3, t2h, t2l, ld3, e3, want);
  }

  // q = B p (q as given to build)
  void apply(cudaStream_t s, const float* p, int* err) {
    tc_pack(s, p, r0 * n, r1, ld1, idx2(r0, 1, n, r0), idx1(r1, (long long)r0 * n), pTh, pTl);
    tc_run(s, g1, err);
    tc_run(s, g2, err);
    if (g3.epi.atomic) QTT_CUDA(cudaMemsetAsync(g3.epi.out, 0, sizeof(float) * (size_t)r0 * n * r1, s));
    tc_run(s, g3, err);
  }
};

// ---------------------------------------------------------------------------
// the solver
// ---------------------------------------------------------------------------
template <typename T>
struct Amen {
  cudaStream_t s;
  Arena& ar;
  const qtt_tensor* A;
  const qtt_tensor* y;
  qtt_tensor* x;
  qtt_tensor* z;
  int D;
  double tol;
  int max_rank, kick, max_sweeps, ndir, restart, cycles, verbose;
  int cg_iters = 40;          // CG iterations per cycle (GMRES keeps restart <= 64)
  bool mixed_local = false;   // FP32 operator inside the local GMRES cycles
  bool tensor_cores = false;  // the FP32 local operator on tcgen05 (3xTF32) at ranks >= 32
  bool tc_always = false;     // ... in every bucket, not only where the autotuner found it faster
  int* tc_err = nullptr;      // device word set by a tensor-core kernel whose bounded wait gave up
  double global_check = 0.0;  // > 0: check the FP64 global residual once max local <= global_check * tol
  bool stall_exit = false;    // stop when two sweeps in a row fail to halve the best max local residual
  // correction solves of the outer refinement: stop as soon as the global
  // residual of outer_u + x for the system outer_A u = outer_f is <= outer_tol
  const qtt_tensor* outer_A = nullptr;
  const qtt_tensor* outer_u = nullptr;
  const qtt_tensor* outer_f = nullptr;
  double outer_tol = 0.0;
  // interfaces: PhiR[k] (bond k), k = 0..D
  std::vector<DBuf<T>> XAX_R, XY_R, ZAX_R, ZY_R;
  DBuf<T> XAX_L, XY_L, ZAX_L, ZY_L, XAX_Ln, XY_Ln, ZAX_Ln, ZY_Ln;
  double* dscal;   // device scratch scalars
  qtt_solve_info* info;
  // FP32 copies of the current core's local operator (mixed precision),
  // made once per core and shared by the Krylov cycles and the truncation
  struct Op32 {
    float* PL = nullptr;
    float* Ak = nullptr;
    float* PR = nullptr;
  } op32;

  Amen(cudaStream_t st, Arena& a) : s(st), ar(a) {}

  int rA(int k) const { return A->r[k]; }
  int ry(int k) const { return y->r[k]; }

  double host_norm(const T* v, size_t n) {
    sumsq<T>(s, v, n, dscal);
    double h;
    QTT_CUDA(cudaMemcpyAsync(&h, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    QTT_CUDA(cudaStreamSynchronize(s));
    return std::sqrt(h);
  }

  // (B x)[a,i,b] with B = PhiL (ra,R0,rc) K_k PhiR (rb,R1,rd), x (rc, n, rd)
  void local_apply(const T* PhiL, int ra, int rc, int k, const T* PhiR, int rb, int rd, const T* xk, T* out, Arena& sc) {
    apply_local<T>(s, sc, PhiL, ra, rc, (const T*)A->core[k], rA(k), A->n[k], rA(k + 1), PhiR, rb, rd, xk, out);
  }

  // g[a,i,b] = PsiL (ra, ryl) y_k (ryl, n, ryr) PsiR (rb, ryr)
  void local_rhs(const T* PsiL, int ra, int k, const T* PsiR, int rb, T* out, Arena& sc) {
    const int n = y->n[k], r0 = ry(k), r1 = ry(k + 1);
    int dL[2] = {ra, r0}, dy[3] = {r0, n, r1};
    T* t = sc.alloc<T>((size_t)ra * n * r1);
    einsum<T>(s, sc, "ac,cid->aid", PsiL, dL, (const T*)y->core[k], dy, t);
    int dt[3] = {ra, n, r1}, dR[2] = {rb, r1};
    einsum<T>(s, sc, "aid,bd->aib", t, dt, PsiR, dR, out);
  }

  // right interface of bond k from bond k+1: Phi[a,A,c] = X[a,i,b] K[A,i,j,B] Y[c,j,d] Phi'[b,B,d]
  void right_XAX(const qtt_tensor* X, const qtt_tensor* Y, int k, const T* Phin, T* out, Arena& sc) {
    const int n = A->n[k], R0 = rA(k), R1 = rA(k + 1);
    const int xa = X->r[k], xb = X->r[k + 1], yc = Y->r[k], yd = Y->r[k + 1];
    int dY[3] = {yc, n, yd}, dP[3] = {xb, R1, yd};
    T* t1 = sc.alloc<T>((size_t)yc * n * xb * R1);
    einsum<T>(s, sc, "cjd,bBd->cjbB", (const T*)Y->core[k], dY, Phin, dP, t1);
    int d1[4] = {yc, n, xb, R1}, dA[4] = {R0, n, n, R1};
    T* t2 = sc.alloc<T>((size_t)yc * xb * R0 * n);
    einsum<T>(s, sc, "cjbB,AijB->cbAi", t1, d1, (const T*)A->core[k], dA, t2);
    int dX[3] = {xa, n, xb}, d2[4] = {yc, xb, R0, n};
    einsum<T>(s, sc, "aib,cbAi->aAc", (const T*)X->core[k], dX, t2, d2, out);
  }

  // left: Phi'[b,B,d] = Phi[a,A,c] X[a,i,b] K[A,i,j,B] Y[c,j,d]
  void left_XAX(const qtt_tensor* X, const qtt_tensor* Y, int k, const T* Phi, T* out, Arena& sc) {
    const int n = A->n[k], R0 = rA(k), R1 = rA(k + 1);
    const int xa = X->r[k], xb = X->r[k + 1], yc = Y->r[k], yd = Y->r[k + 1];
    int dP[3] = {xa, R0, yc}, dX[3] = {xa, n, xb};
    T* t1 = sc.alloc<T>((size_t)R0 * yc * n * xb);
    einsum<T>(s, sc, "aAc,aib->Acib", Phi, dP, (const T*)X->core[k], dX, t1);
    int d1[4] = {R0, yc, n, xb}, dA[4] = {R0, n, n, R1};
    T* t2 = sc.alloc<T>((size_t)yc * xb * n * R1);
    einsum<T>(s, sc, "Acib,AijB->cbjB", t1, d1, (const T*)A->core[k], dA, t2);
    int d2[4] = {yc, xb, n, R1}, dY[3] = {yc, n, yd};
    einsum<T>(s, sc, "cbjB,cjd->bBd", t2, d2, (const T*)Y->core[k], dY, out);
  }

  // Psi[a,c] = X[a,i,b] y[c,i,d] Psi'[b,d]
  void right_XY(const qtt_tensor* X, int k, const T* Psin, T* out, Arena& sc) {
    const int n = y->n[k], xa = X->r[k], xb = X->r[k + 1], c0 = ry(k), c1 = ry(k + 1);
    int dy[3] = {c0, n, c1}, dP[2] = {xb, c1};
    T* t = sc.alloc<T>((size_t)c0 * n * xb);
    einsum<T>(s, sc, "cid,bd->cib", (const T*)y->core[k], dy, Psin, dP, t);
    int dX[3] = {xa, n, xb}, dt[3] = {c0, n, xb};
    einsum<T>(s, sc, "aib,cib->ac", (const T*)X->core[k], dX, t, dt, out);
  }

  void left_XY(const qtt_tensor* X, int k, const T* Psi, T* out, Arena& sc) {
    const int n = y->n[k], xa = X->r[k], xb = X->r[k + 1], c0 = ry(k), c1 = ry(k + 1);
    int dP[2] = {xa, c0}, dX[3] = {xa, n, xb};
    T* t = sc.alloc<T>((size_t)c0 * n * xb);
    einsum<T>(s, sc, "ac,aib->cib", Psi, dP, (const T*)X->core[k], dX, t);
    int dt[3] = {c0, n, xb}, dy[3] = {c0, n, c1};
    einsum<T>(s, sc, "cib,cid->bd", t, dt, (const T*)y->core[k], dy, out);
  }

  void set_one(DBuf<T>& b) {
    b.ensure(1, s);
    fill<T>(s, b.p, 1, T(1));
  }

  void build_right_interfaces() {
    XAX_R.resize(D + 1);
    XY_R.resize(D + 1);
    ZAX_R.resize(D + 1);
    ZY_R.resize(D + 1);
    set_one(XAX_R[D]);
    set_one(XY_R[D]);
    set_one(ZAX_R[D]);
    set_one(ZY_R[D]);
    for (int k = D - 1; k >= 1; --k) {
      Arena sc(s);
      XAX_R[k].ensure((size_t)x->r[k] * rA(k) * x->r[k], s);
      right_XAX(x, x, k, XAX_R[k + 1].p, XAX_R[k].p, sc);
      XY_R[k].ensure((size_t)x->r[k] * ry(k), s);
      right_XY(x, k, XY_R[k + 1].p, XY_R[k].p, sc);
      ZAX_R[k].ensure((size_t)z->r[k] * rA(k) * x->r[k], s);
      right_XAX(z, x, k, ZAX_R[k + 1].p, ZAX_R[k].p, sc);
      ZY_R[k].ensure((size_t)z->r[k] * ry(k), s);
      right_XY(z, k, ZY_R[k + 1].p, ZY_R[k].p, sc);
    }
  }

  // Restarted GMRES on the local operator with the residual of every cycle
  // recomputed in T: x holds the initial guess and receives the solution.
  // With U = float (mixed precision) each cycle runs its Arnoldi process on
  // an FP32 copy of the local operator for the correction equation
  // B d = g - B x, and x += d is accumulated in T (local iterative
  // refinement); with U = T it is plain restarted GMRES.  Returns the final
  // relative residual.
  template <typename U>
  double gmres(int k, const T* PhiL, int r0, const T* PhiR, int r1, const T* g, double gn, T* xk, double rtol) {
    const int n = A->n[k], R0 = rA(k), R1 = rA(k + 1);
    const int N = r0 * n * r1;
    const int m = std::min(restart, N);
    Arena sc(s);
    // operator in U
    const U* PL = reinterpret_cast<const U*>(PhiL);
    const U* PR = reinterpret_cast<const U*>(PhiR);
    const U* Ak = reinterpret_cast<const U*>(A->core[k]);
    if (sizeof(U) != sizeof(T)) {
      if (op32.PL) {   // converted once for this core
        PL = reinterpret_cast<const U*>(op32.PL);
        PR = reinterpret_cast<const U*>(op32.PR);
        Ak = reinterpret_cast<const U*>(op32.Ak);
      } else {
        U* a = sc.alloc<U>((size_t)r0 * R0 * r0);
        convert<T, U>(s, PhiL, a, (size_t)r0 * R0 * r0);
        U* b = sc.alloc<U>((size_t)r1 * R1 * r1);
        convert<T, U>(s, PhiR, b, (size_t)r1 * R1 * r1);
        U* c = sc.alloc<U>((size_t)R0 * n * n * R1);
        convert<T, U>(s, (const T*)A->core[k], c, (size_t)R0 * n * n * R1);
        PL = a;
        PR = b;
        Ak = c;
      }
    }
    U* V = sc.alloc<U>((size_t)N * (m + 1));
    U* w = sc.alloc<U>(N);
    U* hcol = sc.alloc<U>(m + 1);
    U* hcol2 = sc.alloc<U>(m + 1);
    double* H = sc.alloc<double>((size_t)(m + 1) * m);
    double* yv = sc.alloc<double>(m);
    U* yU = sc.alloc<U>(m);
    U* dU = sc.alloc<U>(N);
    T* wT = sc.alloc<T>(N);
    double* dres = sc.alloc<double>(1);
    double* hlast = sc.alloc<double>(1);
    double rel = 1.0;
    for (int cyc = 0; cyc < cycles; ++cyc) {
      Arena it(s);
      // residual in T: wT = g - B x
      local_apply(PhiL, r0, r0, k, PhiR, r1, r1, xk, wT, it);
      axpby<T>(s, N, T(1), g, T(-1), wT);
      double beta = host_norm(wT, N);
      rel = gn > 0 ? beta / gn : beta;
      if (rel <= rtol || beta == 0.0) break;
      QTT_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * (m + 1) * m, s));
      sumsq<T>(s, wT, N, dscal);
      if (sizeof(U) != sizeof(T)) {
        convert<T, U>(s, wT, w, N);
        scale_by_device_kernel<U><<<grid_for(N), 256, 0, s>>>(V, w, N, dscal, nullptr);
      } else {
        scale_by_device_kernel<U><<<grid_for(N), 256, 0, s>>>(V, reinterpret_cast<const U*>(wT), N, dscal, nullptr);
      }
      QTT_CHECK_LAUNCH();
      for (int j = 0; j < m; ++j) {
        Arena ij(s);
        apply_local<U>(s, ij, PL, r0, r0, Ak, R0, n, R1, PR, r1, r1, V + (size_t)N * j, w);
        // classical Gram-Schmidt, twice
        gemm<U>(s, true, false, j + 1, 1, N, U(1), V, N, 0, w, N, 0, U(0), hcol, j + 1, 0);
        gemm<U>(s, false, false, N, 1, j + 1, U(-1), V, N, 0, hcol, j + 1, 0, U(1), w, N, 0);
        gemm<U>(s, true, false, j + 1, 1, N, U(1), V, N, 0, w, N, 0, U(0), hcol2, j + 1, 0);
        gemm<U>(s, false, false, N, 1, j + 1, U(-1), V, N, 0, hcol2, j + 1, 0, U(1), w, N, 0);
        axpby<U>(s, j + 1, U(1), hcol2, U(1), hcol);
        sumsq<U>(s, w, N, dscal);
        scale_by_device_kernel<U><<<grid_for(N), 256, 0, s>>>(V + (size_t)N * (j + 1), w, N, dscal, hlast);
        QTT_CHECK_LAUNCH();
        store_col_kernel<U><<<(m + 128) / 128, 128, 0, s>>>(H, m + 1, j, hcol, j + 1, hlast);
        QTT_CHECK_LAUNCH();
      }
      gmres_lsq_kernel<<<1, 1, 0, s>>>(H, m, beta, yv, dres);
      QTT_CHECK_LAUNCH();
      to_T_kernel<U><<<(m + 127) / 128, 128, 0, s>>>(yv, yU, m);
      QTT_CHECK_LAUNCH();
      gemm<U>(s, false, false, N, 1, m, U(1), V, N, 0, yU, m, 0, U(0), dU, N, 0);
      if (sizeof(U) != sizeof(T)) {
        convert<U, T>(s, dU, wT, N);
        axpby<T>(s, N, T(1), wT, T(1), xk);
      } else {
        axpby<T>(s, N, T(1), reinterpret_cast<const T*>(dU), T(1), xk);
      }
      if (info) info->local_iters += m;
    }
    return rel;
  }

  // Conjugate gradients for a symmetric positive definite local operator,
  // in cycles of `restart` iterations: each cycle recomputes the residual in
  // T, runs CG on B d = g - B x with the operator in U (FP32 when mixed) and
  // adds d to x in T.  All CG scalars stay on the device within a cycle.
  template <typename U>
  double cg(int k, const T* PhiL, int r0, const T* PhiR, int r1, const T* g, double gn, T* xk, double rtol) {
    const int n = A->n[k], R0 = rA(k), R1 = rA(k + 1);
    const int N = r0 * n * r1;
    const int m = std::max(1, cg_iters);
    Arena sc(s);
    const U* PL = reinterpret_cast<const U*>(PhiL);
    const U* PR = reinterpret_cast<const U*>(PhiR);
    const U* Ak = reinterpret_cast<const U*>(A->core[k]);
    if (sizeof(U) != sizeof(T)) {
      if (op32.PL) {   // converted once for this core
        PL = reinterpret_cast<const U*>(op32.PL);
        PR = reinterpret_cast<const U*>(op32.PR);
        Ak = reinterpret_cast<const U*>(op32.Ak);
      } else {
        U* a = sc.alloc<U>((size_t)r0 * R0 * r0);
        convert<T, U>(s, PhiL, a, (size_t)r0 * R0 * r0);
        U* b = sc.alloc<U>((size_t)r1 * R1 * r1);
        convert<T, U>(s, PhiR, b, (size_t)r1 * R1 * r1);
        U* c = sc.alloc<U>((size_t)R0 * n * n * R1);
        convert<T, U>(s, (const T*)A->core[k], c, (size_t)R0 * n * n * R1);
        PL = a;
        PR = b;
        Ak = c;
      }
    }
    U* d = sc.alloc<U>(N);
    U* r = sc.alloc<U>(N);
    U* p = sc.alloc<U>(N);
    U* qv = sc.alloc<U>(N);
    U* z = sc.alloc<U>(N);
    T* wT = sc.alloc<T>(N);
    double* sc4 = sc.alloc<double>(3);       // rz_old, rz_new, pq
    // Jacobi preconditioner: inverse diagonal of the local operator in the
    // interface frames (it scales the frame vectors of different levels)
    U* minv = sc.alloc<U>(N);
    {
      T* dL = sc.alloc<T>((size_t)r0 * R0);
      T* dR = sc.alloc<T>((size_t)r1 * R1);
      T* dK = sc.alloc<T>((size_t)R0 * n * R1);
      diag3_kernel<T><<<(r0 * R0 + 255) / 256, 256, 0, s>>>(PhiL, r0, R0, dL);
      QTT_CHECK_LAUNCH();
      diag3_kernel<T><<<(r1 * R1 + 255) / 256, 256, 0, s>>>(PhiR, r1, R1, dR);
      QTT_CHECK_LAUNCH();
      diagK_kernel<T><<<(R0 * n * R1 + 255) / 256, 256, 0, s>>>((const T*)A->core[k], R0, n, R1, dK);
      QTT_CHECK_LAUNCH();
      int e1[2] = {r0, R0}, e2[3] = {R0, n, R1}, e3[3] = {r0, n, R1}, e4[2] = {r1, R1};
      T* t = sc.alloc<T>((size_t)r0 * n * R1);
      einsum<T>(s, sc, "aA,AiB->aiB", dL, e1, dK, e2, t);
      T* dg = sc.alloc<T>(N);
      einsum<T>(s, sc, "aiB,bB->aib", t, e3, dR, e4, dg);
      inv_diag_kernel<T, U><<<(N + 255) / 256, 256, 0, s>>>(dg, minv, N);
      QTT_CHECK_LAUNCH();
    }
    const bool tc_ok = sizeof(U) == 4 && sizeof(T) == 8 && tensor_cores && op32.PL && tc_err && r0 >= 32 &&
                       r1 >= 32 && tc_available() && persistent_cg_grid() > 0;
    const int choice = tc_ok ? (tc_always ? 1 : tune_choice(r0, r1)) : 0;
    const bool use_tc = tc_ok && (choice == 1 || choice == 2);
    const bool timing = tc_ok && (choice == 2 || choice == 3);
    cudaEvent_t tev0 = nullptr, tev1 = nullptr;
    double tune_ms = 0.0;
    long long tune_iters = 0;
    if (timing) {
      QTT_CUDA(cudaEventCreate(&tev0));
      QTT_CUDA(cudaEventCreate(&tev1));
    }
    TcLocalOp tl;
    if (use_tc)
      tl.build(s, sc, reinterpret_cast<const float*>(PL), reinterpret_cast<const float*>(Ak),
               reinterpret_cast<const float*>(PR), r0, n, r1, R0, R1, reinterpret_cast<float*>(qv));
    double rel = 1.0, prev = -1.0;
    for (int cyc = 0; cyc < cycles; ++cyc) {
      Arena it(s);
      local_apply(PhiL, r0, r0, k, PhiR, r1, r1, xk, wT, it);
      axpby<T>(s, N, T(1), g, T(-1), wT);     // residual in T
      double beta = host_norm(wT, N);
      rel = gn > 0 ? beta / gn : beta;
      if (rel <= rtol || beta == 0.0) break;
      if (sizeof(U) != sizeof(T) && prev > 0.0 && rel > 0.9 * prev) break;   // FP32 cycles stopped gaining
      prev = rel;
      convert<T, U>(s, wT, r, N);
      precond_kernel<U><<<grid_for(N), 256, 0, s>>>(p, minv, r, N);   // p = z = M^-1 r
      QTT_CHECK_LAUNCH();
      QTT_CUDA(cudaMemsetAsync(d, 0, sizeof(U) * N, s));
      double* rr_old = sc4;
      double* rr_new = sc4 + 1;
      double* pq = sc4 + 2;
      dotp<U>(s, r, p, N, rr_old);
      if (timing) QTT_CUDA(cudaEventRecord(tev0, s));
      if (use_tc) {
        // every iteration on the tensor cores: B p by three 3xTF32 GEMMs,
        // the CG scalars on the device
        for (int j = 0; j < m; ++j) {
          tl.apply(s, reinterpret_cast<const float*>(p), tc_err);
          dotp<U>(s, p, qv, N, pq);
          cg_step_kernel<U><<<grid_for(N), 256, 0, s>>>(d, r, p, qv, rr_old, pq, N);
          QTT_CHECK_LAUNCH();
          precond_kernel<U><<<grid_for(N), 256, 0, s>>>(z, minv, r, N);
          QTT_CHECK_LAUNCH();
          dotp<U>(s, r, z, N, rr_new);
          cg_dir_kernel<U><<<grid_for(N), 256, 0, s>>>(p, z, rr_new, rr_old, N);
          QTT_CHECK_LAUNCH();
          std::swap(rr_old, rr_new);
        }
        int herr = 0;
        QTT_CUDA(cudaMemcpyAsync(&herr, tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        QTT_CUDA(cudaStreamSynchronize(s));
        if (herr != 0) throw QttError(QTT_ETIMEOUT, "local CG: a tensor-core kernel's bounded wait gave up");
      } else if (sizeof(U) == 4 && persistent_cg_grid() > 0) {
        // all m iterations in one cooperative launch
        const int grid = persistent_cg_grid();
        PcgArgs pa{};
        int dx[3] = {r0, n, r1}, dR[3] = {r1, R1, r1}, d1[4] = {r0, n, r1, R1}, dA[4] = {R0, n, n, R1};
        int dL[3] = {r0, R0, r0}, d2[4] = {r0, r1, R0, n};
        bool ok = plan_contract("cjd,bBd->cjbB", dx, dR, 4, 0, pa.c1) &&
                  plan_contract("cjbB,AijB->cbAi", d1, dA, 4, 0, pa.c2) &&
                  plan_contract("aAc,cbAi->aib", dL, d2, 4, grid, pa.c3);
        QTT_REQUIRE(ok, "persistent CG: contraction plan failed");
        float* t1 = sc.alloc<float>((size_t)r0 * n * r1 * R1);
        float* t2 = sc.alloc<float>((size_t)r0 * r1 * R0 * n);
        QTT_CUDA(cudaMemsetAsync(sc4 + 1, 0, 2 * sizeof(double), s));
        pa.PL = reinterpret_cast<const float*>(PL);
        pa.Ak = reinterpret_cast<const float*>(Ak);
        pa.PR = reinterpret_cast<const float*>(PR);
        pa.minv = reinterpret_cast<const float*>(minv);
        pa.t1 = t1;
        pa.t2 = t2;
        pa.d = reinterpret_cast<float*>(d);
        pa.r = reinterpret_cast<float*>(r);
        pa.p = reinterpret_cast<float*>(p);
        pa.q = reinterpret_cast<float*>(qv);
        pa.acc = sc4;
        pa.N = N;
        pa.iters = m;
        void* kargs[] = {&pa};
        ProfToken pt = prof_begin(PROF_PCG, s);
        QTT_CUDA(cudaLaunchCooperativeKernel((void*)pcg_kernel, grid, 256, kargs, 0, s));
        count_launch();
        if (pt.ev) {
          // per iteration: the three contractions of B p, three dot products
          // and the d, r, p updates; bytes: the three operator factors read
          // once (they stay in L2 across iterations, so this is per launch),
          // plus the vectors and contraction intermediates written and read
          const double fl = 2.0 * ((double)r0 * n * r1 * R1 * r1 + (double)r0 * r1 * R0 * n * n * R1 +
                                   (double)r0 * R0 * r0 * r1 * n) + 16.0 * N;
          const double ops = (double)r0 * R0 * r0 + (double)R0 * n * n * R1 + (double)r1 * R1 * r1;
          const double vec = 2.0 * ((double)r0 * n * r1 * R1 + (double)r0 * r1 * R0 * n) + 12.0 * N;
          prof_end(pt, s, fl * m, 4.0 * (ops + vec * m));
        }
      } else {
        for (int j = 0; j < m; ++j) {
          Arena ij(s);
          apply_local<U>(s, ij, PL, r0, r0, Ak, R0, n, R1, PR, r1, r1, p, qv);
          dotp<U>(s, p, qv, N, pq);
          cg_step_kernel<U><<<grid_for(N), 256, 0, s>>>(d, r, p, qv, rr_old, pq, N);
          QTT_CHECK_LAUNCH();
          precond_kernel<U><<<grid_for(N), 256, 0, s>>>(z, minv, r, N);
          QTT_CHECK_LAUNCH();
          dotp<U>(s, r, z, N, rr_new);
          cg_dir_kernel<U><<<grid_for(N), 256, 0, s>>>(p, z, rr_new, rr_old, N);
          QTT_CHECK_LAUNCH();
          std::swap(rr_old, rr_new);
        }
      }
      if (timing) {
        QTT_CUDA(cudaEventRecord(tev1, s));
        QTT_CUDA(cudaEventSynchronize(tev1));
        float ms = 0.f;
        QTT_CUDA(cudaEventElapsedTime(&ms, tev0, tev1));
        tune_ms += ms;
        tune_iters += m;
      }
      if (sizeof(U) != sizeof(T)) {
        convert<U, T>(s, d, wT, N);
        axpby<T>(s, N, T(1), wT, T(1), xk);
      } else {
        axpby<T>(s, N, T(1), reinterpret_cast<const T*>(d), T(1), xk);
      }
      if (info) info->local_iters += m;
    }
    if (timing) {
      if (tune_iters > 0) tune_record(r0, r1, use_tc, 1e3 * tune_ms / (double)tune_iters);
      cudaEventDestroy(tev0);
      cudaEventDestroy(tev1);
    }
    return rel;
  }

  double local_residual(int k, const T* PhiL, int r0, const T* PhiR, int r1, const T* g, double gn, const T* xk,
                        T* keep = nullptr) {
    const int N = r0 * A->n[k] * r1;
    Arena sc(s);
    T* w = keep ? keep : sc.alloc<T>(N);
    local_apply(PhiL, r0, r0, k, PhiR, r1, r1, xk, w, sc);
    axpby<T>(s, N, T(-1), g, T(1), w);      // w = B x - g
    double rn = host_norm(w, N);
    return gn > 0 ? rn / gn : rn;
  }

  // ||B t - w|| / gn with t applied in FP32 (the FP32 operator of op32) and
  // w = B x_sol - g in FP64: the local residual of x_sol - t.
  double tail_residual32(int k, int r0, int r1, const float* t32, const T* w, double gn, Arena& sc) {
    const int n = A->n[k], N = r0 * n * r1;
    float* bt = sc.alloc<float>(N);
    apply_local<float>(s, sc, op32.PL, r0, r0, op32.Ak, rA(k), n, rA(k + 1), op32.PR, r1, r1, t32, bt);
    QTT_CUDA(cudaMemsetAsync(dscal, 0, sizeof(double), s));
    diff_sumsq_kernel<T><<<std::min(grid_for(N), 2 * num_sms()), 256, 0, s>>>(bt, w, N, dscal);
    QTT_CHECK_LAUNCH();
    double h;
    QTT_CUDA(cudaMemcpyAsync(&h, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
    QTT_CUDA(cudaStreamSynchronize(s));
    return gn > 0 ? std::sqrt(h) / gn : std::sqrt(h);
  }

  void ensure_core(qtt_tensor* t, int k, size_t elems) { tensor_reserve(t, k, elems, s); }

  int run() {
    // With the FP64 global check deciding convergence, the sweeps truncate
    // and solve at a 4x tighter local level: truncating every core at
    // tol / sqrt(D) in the local residual norm leaves a global residual up
    // to a few times tol, where the sweeps stagnate.
    const bool global_stop = sizeof(T) == 8 && global_check > 0;
    const double tloc = global_stop ? 0.25 * tol : tol;
    const double delta = tloc / std::sqrt((double)D);
    int status = QTT_ENOCONV;
    const auto t_start = std::chrono::steady_clock::now();
    double best_res = 1e300, checked_at = 1e300;
    int stalled = 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
      {
        Arena sc(s);
        right_orthogonalize<T>(s, sc, x, 0);
        right_orthogonalize<T>(s, sc, z, 0);
      }
      build_right_interfaces();
      set_one(XAX_L);
      set_one(XY_L);
      set_one(ZAX_L);
      set_one(ZY_L);
      double max_res = 0.0;
      for (int k = 0; k < D; ++k) {
        Arena sc(s);
        const int r0 = x->r[k], r1 = x->r[k + 1], n = A->n[k];
        const int N = r0 * n * r1;
        const T* PhiR = XAX_R[k + 1].p;
        T* g = sc.alloc<T>(N);
        local_rhs(XY_L.p, r0, k, XY_R[k + 1].p, r1, g, sc);
        const double gn = host_norm(g, N);
        T* xk = (T*)x->core[k];
        const double res = local_residual(k, XAX_L.p, r0, PhiR, r1, g, gn, xk);
        max_res = std::max(max_res, res);
        // local solve
        T* sol = sc.alloc<T>(N);
        if (N <= ndir) {
          T* Bm = sc.alloc<T>((size_t)N * N);
          const int R0 = rA(k), R1 = rA(k + 1);
          int dL[3] = {r0, R0, r0}, dA[4] = {R0, n, n, R1};
          T* t = sc.alloc<T>((size_t)r0 * r0 * n * n * R1);
          einsum<T>(s, sc, "aAc,AijB->acijB", XAX_L.p, dL, (const T*)A->core[k], dA, t);
          int dt[5] = {r0, r0, n, n, R1}, dR[3] = {r1, R1, r1};
          einsum<T>(s, sc, "acijB,bBd->aibcjd", t, dt, PhiR, dR, Bm);
          QTT_CUDA(cudaMemcpyAsync(sol, g, sizeof(T) * N, cudaMemcpyDeviceToDevice, s));
          int* dinfo = sc.alloc<int>(1);
          lu_solve<T>(s, sc, N, Bm, N, sol, N, 1, dinfo);
        } else {
          QTT_CUDA(cudaMemcpyAsync(sol, xk, sizeof(T) * N, cudaMemcpyDeviceToDevice, s));
          if (mixed_local && sizeof(T) == 8) {
            const int R0 = rA(k), R1 = rA(k + 1);
            op32.PL = sc.alloc<float>((size_t)r0 * R0 * r0);
            convert<T, float>(s, XAX_L.p, op32.PL, (size_t)r0 * R0 * r0);
            op32.PR = sc.alloc<float>((size_t)r1 * R1 * r1);
            convert<T, float>(s, PhiR, op32.PR, (size_t)r1 * R1 * r1);
            op32.Ak = sc.alloc<float>((size_t)R0 * n * n * R1);
            convert<T, float>(s, (const T*)A->core[k], op32.Ak, (size_t)R0 * n * n * R1);
          }
          if (A->sym) {
            if (mixed_local && sizeof(T) == 8) cg<float>(k, XAX_L.p, r0, PhiR, r1, g, gn, sol, delta);
            else cg<T>(k, XAX_L.p, r0, PhiR, r1, g, gn, sol, delta);
          } else if (mixed_local && sizeof(T) == 8) gmres<float>(k, XAX_L.p, r0, PhiR, r1, g, gn, sol, delta);
          else gmres<T>(k, XAX_L.p, r0, PhiR, r1, g, gn, sol, delta);
        }
        if (info) info->local_solves += 1;
        if (k == D - 1) {
          QTT_CUDA(cudaMemcpyAsync(xk, sol, sizeof(T) * N, cudaMemcpyDeviceToDevice, s));
          op32 = Op32{};
          break;
        }
        T* wsol = sc.alloc<T>(N);
        const double res_sol = local_residual(k, XAX_L.p, r0, PhiR, r1, g, gn, sol, wsol);
        // SVD of the left unfolding (r0 n) x r1
        const int rows = r0 * n, kk = std::min(rows, r1);
        T* Acp = sc.alloc<T>(N);
        QTT_CUDA(cudaMemcpyAsync(Acp, sol, sizeof(T) * N, cudaMemcpyDeviceToDevice, s));
        T* U = sc.alloc<T>((size_t)rows * kk);
        T* S = sc.alloc<T>(kk);
        T* Vt = sc.alloc<T>((size_t)kk * r1);
        svd<T>(s, sc, rows, r1, Acp, rows, U, rows, S, Vt, kk);
        // residual-norm truncation by bisection
        const double thr = std::max(delta, 2.0 * res_sol);
        int lo = 1, hi = kk;
        T* cand = sc.alloc<T>(N);
        T* SV = sc.alloc<T>((size_t)kk * r1);
        scale_rows_kernel<T><<<grid_for((long long)kk * r1), 256, 0, s>>>(kk, r1, Vt, kk, S, SV, kk);
        QTT_CHECK_LAUNCH();
        if (op32.PL) {
          // mixed precision: the residual of x_sol - tail_m is w_sol - B tail_m
          // with w_sol = B x_sol - g exact in FP64 and only the small tail
          // applied in FP32 (an FP32 error relative to B tail_m moves the
          // chosen rank by one at most; the FP64 global check decides)
          float* U32 = sc.alloc<float>((size_t)rows * kk);
          float* SV32 = sc.alloc<float>((size_t)kk * r1);
          float* tail = sc.alloc<float>(N);
          convert<T, float>(s, U, U32, (size_t)rows * kk);
          convert<T, float>(s, SV, SV32, (size_t)kk * r1);
          while (lo < hi) {
            int mid = (lo + hi) / 2;
            Arena bs(s);
            gemm<float>(s, false, false, rows, r1, kk - mid, 1.f, U32 + (size_t)rows * mid, rows, 0, SV32 + mid, kk,
                        0, 0.f, tail, rows, 0);
            if (tail_residual32(k, r0, r1, tail, wsol, gn, bs) <= thr) hi = mid;
            else lo = mid + 1;
          }
        } else {
          while (lo < hi) {
            int mid = (lo + hi) / 2;
            gemm<T>(s, false, false, rows, r1, mid, T(1), U, rows, 0, SV, kk, 0, T(0), cand, rows, 0);
            if (local_residual(k, XAX_L.p, r0, PhiR, r1, g, gn, cand) <= thr) hi = mid;
            else lo = mid + 1;
          }
        }
        int rk = hi;
        if (max_rank > 0) rk = std::min(rk, std::max(1, max_rank - kick));
        // truncated core xt = U_rk S V_rk^T
        gemm<T>(s, false, false, rows, r1, rk, T(1), U, rows, 0, SV, kk, 0, T(0), cand, rows, 0);
        // new residual-proxy core
        const int rz0 = z->r[k], rz1 = z->r[k + 1];
        T* zres = sc.alloc<T>((size_t)rz0 * n * rz1);
        T* tmp = sc.alloc<T>((size_t)rz0 * n * rz1);
        local_rhs(ZY_L.p, rz0, k, ZY_R[k + 1].p, rz1, zres, sc);
        local_apply(ZAX_L.p, rz0, r0, k, ZAX_R[k + 1].p, rz1, r1, cand, tmp, sc);
        axpby<T>(s, (size_t)rz0 * n * rz1, T(-1), tmp, T(1), zres);
        const int zrows = rz0 * n, zk = std::min(zrows, rz1);
        T* Qz = sc.alloc<T>((size_t)zrows * zk);
        T* Rz = sc.alloc<T>((size_t)zk * rz1);
        qr<T>(s, sc, zrows, rz1, zres, zrows, Qz, zrows, Rz, zk);
        // enrichment block: residual on x's left and z's right interfaces
        T* enr = sc.alloc<T>((size_t)r0 * n * rz1);
        T* tmp2 = sc.alloc<T>((size_t)r0 * n * rz1);
        local_rhs(XY_L.p, r0, k, ZY_R[k + 1].p, rz1, enr, sc);
        local_apply(XAX_L.p, r0, r0, k, ZAX_R[k + 1].p, rz1, r1, cand, tmp2, sc);
        axpby<T>(s, (size_t)r0 * n * rz1, T(-1), tmp2, T(1), enr);
        // Uaug = [U_rk, enr]  ->  Q R
        const int ca = rk + rz1, nk = std::min(rows, ca);
        T* Uaug = sc.alloc<T>((size_t)rows * ca);
        QTT_CUDA(cudaMemcpyAsync(Uaug, U, sizeof(T) * rows * rk, cudaMemcpyDeviceToDevice, s));
        QTT_CUDA(cudaMemcpyAsync(Uaug + (size_t)rows * rk, enr, sizeof(T) * rows * rz1, cudaMemcpyDeviceToDevice, s));
        T* Q = sc.alloc<T>((size_t)rows * nk);
        T* Rq = sc.alloc<T>((size_t)nk * ca);
        qr<T>(s, sc, rows, ca, Uaug, rows, Q, rows, Rq, nk);
        // carry = R[:, :rk] (S V^T)[:rk, :]   (nk x r1)
        T* carry = sc.alloc<T>((size_t)nk * r1);
        gemm<T>(s, false, false, nk, r1, rk, T(1), Rq, nk, 0, SV, kk, 0, T(0), carry, nk, 0);
        // next core <- carry * x_{k+1}
        const int n2 = A->n[k + 1], r2 = x->r[k + 2];
        T* nxt = sc.alloc<T>((size_t)nk * n2 * r2);
        gemm<T>(s, false, false, nk, n2 * r2, r1, T(1), carry, nk, 0, (const T*)x->core[k + 1], r1, 0, T(0), nxt, nk,
                0);
        ensure_core(x, k, (size_t)rows * nk);
        ensure_core(x, k + 1, (size_t)nk * n2 * r2);
        QTT_CUDA(cudaMemcpyAsync(x->core[k], Q, sizeof(T) * rows * nk, cudaMemcpyDeviceToDevice, s));
        QTT_CUDA(cudaMemcpyAsync(x->core[k + 1], nxt, sizeof(T) * nk * n2 * r2, cudaMemcpyDeviceToDevice, s));
        x->r[k + 1] = nk;
        // z core k <- Qz; next z core keeps its leading zk rows
        const int zn2 = z->n[k + 1], zr2 = z->r[k + 2];
        QTT_CUDA(cudaMemcpyAsync(z->core[k], Qz, sizeof(T) * zrows * zk, cudaMemcpyDeviceToDevice, s));
        if (zk != rz1) {
          T* znext = sc.alloc<T>((size_t)zk * zn2 * zr2);
          copy2d<T>(s, zk, zn2 * zr2, (const T*)z->core[k + 1], rz1, znext, zk);
          QTT_CUDA(cudaMemcpyAsync(z->core[k + 1], znext, sizeof(T) * zk * zn2 * zr2, cudaMemcpyDeviceToDevice, s));
        }
        z->r[k + 1] = zk;
        // left interfaces
        XAX_Ln.ensure((size_t)nk * rA(k + 1) * nk, s);
        left_XAX(x, x, k, XAX_L.p, XAX_Ln.p, sc);
        XY_Ln.ensure((size_t)nk * ry(k + 1), s);
        left_XY(x, k, XY_L.p, XY_Ln.p, sc);
        ZAX_Ln.ensure((size_t)zk * rA(k + 1) * nk, s);
        left_XAX(z, x, k, ZAX_L.p, ZAX_Ln.p, sc);
        ZY_Ln.ensure((size_t)zk * ry(k + 1), s);
        left_XY(z, k, ZY_L.p, ZY_Ln.p, sc);
        XAX_L.swap(XAX_Ln);
        XY_L.swap(XY_Ln);
        ZAX_L.swap(ZAX_Ln);
        ZY_L.swap(ZY_Ln);
        op32 = Op32{};
      }
      if (info) {
        info->sweeps += 1;
        info->max_local_res = max_res;
      }
      if (verbose) {
        QTT_CUDA(cudaStreamSynchronize(s));
        fprintf(stderr, "[qtt_solve %s %.2fs] sweep %d max local res %.3e ranks", sizeof(T) == 8 ? "f64" : "f32",
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count(), sweep + 1, max_res);
        for (int k = 0; k <= D; ++k) fprintf(stderr, " %d", x->r[k]);
        fprintf(stderr, "\n");
      }
      if (max_res <= tloc) {
        status = QTT_OK;
        break;
      }
      // a correction good enough for the outer system ends its solve early
      // (affordable when the global residual is applied in full format)
      if (outer_u && sweep >= 2 && has_fe_operator(outer_A)) {
        const double rel = timed_residual64(s, outer_A, outer_u, outer_f, info, x);
        if (verbose)
          fprintf(stderr, "[qtt_solve] sweep %d: outer residual with this correction %.3e\n", sweep + 1, rel);
        if (rel <= outer_tol) {
          status = QTT_OK;
          break;
        }
      }
      // Near the tolerance the local residuals can hover above it while the
      // global one is already below (the local ones are projections of the
      // last iterate's residual, measured before each core's update): once
      // they are within global_check x tol, the FP64 global residual decides.
      // It is measured again only after the local residuals have halved.
      if (sizeof(T) == 8 && global_check > 0 && max_res <= global_check * tol && max_res <= 0.5 * checked_at) {
        checked_at = max_res;
        const double rel = timed_residual64(s, A, x, y, info);
        if (info) info->rel_residual = rel;
        if (verbose)
          fprintf(stderr, "[qtt_solve f64 %.2fs] sweep %d global FP64 rel residual %.3e\n",
                  std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count(), sweep + 1, rel);
        if (rel <= tol) {
          status = QTT_OK;
          break;
        }
      }
      // At large L the local systems are too ill-conditioned for the local
      // Krylov solves to reach tol, and the sweeps stall a little above it;
      // the caller's outer refinement takes over from there.
      // (counted only within 100 x tol: farther out, the residual can stay
      // level for a few sweeps while the ranks grow)
      if (max_res <= 0.5 * best_res) {
        best_res = max_res;
        stalled = 0;
      } else if (stall_exit && max_res <= 1e2 * tol && ++stalled >= 2) {
        if (verbose) fprintf(stderr, "[qtt_solve] sweeps stalled at max local res %.3e\n", max_res);
        break;
      }
    }
    return status;
  }
};

template <typename S, typename D>
__global__ void cvt_kernel(const S* a, D* b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = (D)a[i];
}

Tptr default_x0(cudaStream_t s, const qtt_tensor* f, int prec) {
  std::vector<int> r(f->d + 1, 1);
  auto x = own(tensor_alloc(f->d, f->n, nullptr, r.data(), prec, 0));
  for (int k = 0; k < f->d; ++k) {
    if (prec == QTT_F64) fill<double>(s, (double*)x->core[k], f->n[k], 1.0);
    else fill<float>(s, (float*)x->core[k], f->n[k], 1.0f);
  }
  return x;
}

Tptr default_z0(cudaStream_t s, const qtt_tensor* f, int rho, int prec) {
  std::vector<int> r(f->d + 1, rho);
  r[0] = r[f->d] = 1;
  auto z = own(tensor_alloc(f->d, f->n, nullptr, r.data(), prec, 0));
  for (int k = 0; k < f->d; ++k) {
    long long e = (long long)core_elems(z.get(), k);
    if (prec == QTT_F64) proxy_kernel<double><<<grid_for(e), 256, 0, s>>>((double*)z->core[k], e, k);
    else proxy_kernel<float><<<grid_for(e), 256, 0, s>>>((float*)z->core[k], e, k);
    QTT_CHECK_LAUNCH();
  }
  return z;
}

struct OuterCheck {
  const qtt_tensor* u = nullptr;
  const qtt_tensor* f = nullptr;
  double tol = 0.0;
};

template <typename T>
int amen_run(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* f, qtt_tensor* x, qtt_tensor* z, double tol,
             const qtt_solve_opts& o, qtt_solve_info* info, bool mixed_local = false, bool stall_exit = false,
             double global_check = 30.0, OuterCheck outer = OuterCheck{}) {
  Arena ar(s);
  Amen<T> am(s, ar);
  am.A = K;
  am.y = f;
  am.x = x;
  am.z = z;
  am.D = K->d;
  am.tol = tol;
  am.max_rank = o.max_rank > 0 ? o.max_rank : 512;
  am.kick = z->r[1];
  am.max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : 30;
  am.ndir = o.local_direct_max > 0 ? o.local_direct_max : 2048;
  am.restart = std::min(o.local_restart > 0 ? o.local_restart : 40, 64);   // GMRES Hessenberg storage
  am.cg_iters = std::min(o.local_restart > 0 ? o.local_restart : 40, 1000);
  am.cycles = o.local_max_cycles > 0 ? o.local_max_cycles : 20;
  am.verbose = o.verbose;
  am.info = info;
  am.mixed_local = mixed_local;
  am.tensor_cores = mixed_local && o.tensor_cores >= 0;
  am.tc_always = o.tensor_cores > 0;
  if (am.tensor_cores) {
    am.tc_err = ar.alloc<int>(1);
    QTT_CUDA(cudaMemsetAsync(am.tc_err, 0, sizeof(int), s));
  }
  am.global_check = global_check;
  am.stall_exit = stall_exit;
  if (outer.u) {
    am.outer_A = K;
    am.outer_u = outer.u;
    am.outer_f = outer.f;
    am.outer_tol = outer.tol;
  }
  am.dscal = ar.alloc<double>(4);
  int rc = am.run();
  QTT_CUDA(cudaStreamSynchronize(s));
  return rc;
}

double erank_of(const qtt_tensor* x) {
  const int d = x->d;
  if (d == 1) return 1.0;
  double S = 0;
  for (int k = 0; k < d; ++k) S += (double)core_elems(x, k);
  double a = 0, b = (double)x->n[0] * x->m[0] + (double)x->n[d - 1] * x->m[d - 1];
  for (int k = 1; k < d - 1; ++k) a += (double)x->n[k] * x->m[k];
  if (a == 0) return S / b;
  return (-b + std::sqrt(b * b + 4 * a * S)) / (2 * a);
}

}  // namespace

// fraction of the GPU a solve issued from this thread may occupy with one
// cooperative launch (1/n of the SMs; batched workers set n = worker count)
void set_gpu_share(int n) { g_gpu_share = std::max(1, n); }

// FP64 relative residual ||f - K u|| / ||f||.  The product K u is formed
// exactly by the QTT matvec in FP64 (ranks R r).  When the full vector fits
// (<= 2^28 entries) the norm is taken after expanding f - K u to full format
// (one FP64 GEMM of the left and right partial expansions: O(N R r) flops,
// exact up to rounding); otherwise the sum is normed by FP64 left
// orthogonalisation (O(D (R r)^3) flops).
double residual64(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f) {
  Arena ar(s);
  auto Ku = own(product<double>(s, K, u));
  auto r = own(tt_sum<double>(s, 1.0, f, -1.0, Ku.get()));
  long long total = 1;
  for (int k = 0; k < r->d; ++k) total *= r->n[k];
  if (total <= (1LL << 28)) {
    double* full = ar.alloc<double>(total);
    to_full<double>(s, ar, r.get(), full, (size_t)total, QTT_ORDER_Z_BLOCK);
    double* dv = ar.alloc<double>(1);
    sumsq<double>(s, full, (size_t)total, dv);
    double rn2 = 0;
    QTT_CUDA(cudaMemcpyAsync(&rn2, dv, sizeof(double), cudaMemcpyDeviceToHost, s));
    double* ff = ar.alloc<double>(total);
    to_full<double>(s, ar, f, ff, (size_t)total, QTT_ORDER_Z_BLOCK);
    double* df = ar.alloc<double>(1);
    sumsq<double>(s, ff, (size_t)total, df);
    double fn2 = 0;
    QTT_CUDA(cudaMemcpyAsync(&fn2, df, sizeof(double), cudaMemcpyDeviceToHost, s));
    QTT_CUDA(cudaStreamSynchronize(s));
    return fn2 > 0 ? std::sqrt(rn2 / fn2) : std::sqrt(rn2);
  }
  double rn = norm<double>(s, ar, r.get());
  double fn = norm<double>(s, ar, f);
  return fn > 0 ? rn / fn : rn;
}

int solve(const qtt_tensor* K, const qtt_tensor* f, const qtt_tensor* x0, const qtt_tensor* z0,
          const qtt_solve_opts* opts, qtt_tensor** xout, qtt_solve_info* info, cudaStream_t s) {
  QTT_REQUIRE(K && f && opts && xout, "qtt_solve: null argument");
  QTT_REQUIRE(K->is_matrix && !f->is_matrix && K->d == f->d, "qtt_solve: K must be an MPO and f an MPS of equal length");
  for (int k = 0; k < K->d; ++k)
    QTT_REQUIRE(K->n[k] == f->n[k] && K->m[k] == f->n[k], "qtt_solve: mode sizes of K and f differ");
  QTT_REQUIRE(opts->tol > 0, "qtt_solve: tol must be positive");
  qtt_solve_opts o = *opts;
  qtt_solve_info local{};
  qtt_solve_info* inf = info ? info : &local;
  std::memset(inf, 0, sizeof(*inf));
  const int rho = o.kick_rank > 0 ? o.kick_rank : 8;
  int rc = QTT_OK;
  if (o.precision == QTT_F32) {
    Tptr Kc = own(nullptr), fc = own(nullptr);
    const qtt_tensor* Ku = K;
    const qtt_tensor* fu = f;
    if (K->prec != QTT_F32) { Kc = own(tensor_clone(K, QTT_F32, s)); Ku = Kc.get(); }
    if (f->prec != QTT_F32) { fc = own(tensor_clone(f, QTT_F32, s)); fu = fc.get(); }
    Tptr x = x0 ? own(tensor_clone(x0, QTT_F32, s)) : default_x0(s, f, QTT_F32);
    Tptr z = z0 ? own(tensor_clone(z0, QTT_F32, s)) : default_z0(s, f, rho, QTT_F32);
    rc = amen_run<float>(s, Ku, fu, x.get(), z.get(), o.tol, o, inf);
    *xout = x.release();
  } else {
    QTT_REQUIRE(o.precision == QTT_F64 || o.precision == QTT_MIXED, "qtt_solve: unknown precision");
    QTT_REQUIRE(K->prec == QTT_F64 && f->prec == QTT_F64, "qtt_solve: FP64 and mixed solves need FP64 K and f");
    // Sweeps with FP64 interfaces and local residuals; with QTT_MIXED the
    // Krylov cycles of every local solve apply an FP32 copy of the local
    // operator (local iterative refinement).  The FP64 global residual
    // r = f - K u (QTT matvec in FP64) decides.  When the sweeps stall above
    // tol, r is rounded in FP64 (randomized, round_residual_rand), K d = r is
    // solved the same way to the inner tolerance, and u <- u + d (rounded at
    // the level of FP64 noise only).
    const bool mixed = o.precision == QTT_MIXED;
    const double inner = o.inner_tol > 0 ? o.inner_tol : 1e-3;
    const int refine_max = o.refine_max > 0 ? o.refine_max : (o.refine_max < 0 ? 0 : 6);
    Tptr u = x0 ? own(tensor_clone(x0, QTT_F64, s)) : default_x0(s, f, QTT_F64);
    Tptr z = z0 ? own(tensor_clone(z0, QTT_F64, s)) : default_z0(s, f, rho, QTT_F64);
    rc = amen_run<double>(s, K, f, u.get(), z.get(), o.tol, o, inf, mixed, refine_max > 0);
    double fnorm = -1.0, prev_rel = -1.0;
    bool qtt_residual_stalled = false;
    for (int it = 0;; ++it) {
      // a passing in-sweep check stops the sweeps at once, so a stored value
      // <= tol is the final iterate's residual; otherwise measure it now
      const double rel = (it == 0 && rc == QTT_OK && inf->rel_residual > 0 && inf->rel_residual <= o.tol)
                             ? inf->rel_residual
                             : timed_residual64(s, K, u.get(), f, inf);
      inf->rel_residual = rel;
      // a correction that did not halve the residual: the residual formed
      // in QTT arithmetic has lost what the correction needs
      if (prev_rel > 0.0 && rel > 0.5 * prev_rel) qtt_residual_stalled = true;
      prev_rel = rel;
      if (o.verbose) fprintf(stderr, "[qtt_solve] check %d: FP64 rel residual %.3e\n", it, rel);
      if (rel <= o.tol || it >= refine_max) {
        rc = rel <= o.tol ? QTT_OK : QTT_ENOCONV;
        break;
      }
      const auto t_ref = std::chrono::steady_clock::now();
      if (fnorm < 0) {
        Arena ar(s);
        fnorm = norm<double>(s, ar, f);
      }
      Tptr r = own(nullptr);
      if (has_fe_operator(K) && (rel <= kFeResidualBelow || qtt_residual_stalled)) {
        // Near the FP64 floor the residual's low-frequency part -- the one
        // that carries the error, K^-1 r -- is a small fraction of ||r||
        // and lost to cancellation when f - K u is formed inside the QTT
        // cores; formed element by element and TT-SVD-compressed it keeps
        // it (a rank-16 TT-SVD of the L = 10 plate's residual already
        // carries all but 3 % of K^-1 r)
        r = own(residual_fe_tt(s, K, u.get(), f, std::min(1e-2, inner), kFeResidualRank, nullptr));
        if (o.verbose) {
          int rr = 1;
          for (int k = 0; k <= r->d; ++k) rr = std::max(rr, r->r[k]);
          fprintf(stderr, "[qtt_solve] refinement %d: residual formed in full format, TT-SVD max rank %d\n", it + 1,
                  rr);
        }
      } else {
        int mr = 1;
        for (int k = 0; k <= u->d; ++k) mr = std::max(mr, u->r[k]);
        const int ell = std::min(512, std::max(64, 4 * mr + 16));
        double kept = 0.0;
        r = own(round_residual_rand(s, K, u.get(), f, ell, 0x5eed0000ULL + (unsigned long long)it, &kept));
        if (o.verbose) {
          const double full = rel * fnorm, frac = full > 0 ? kept / full : 1.0;
          fprintf(stderr, "[qtt_solve] refinement %d: residual sketched at rank %d, relative error %.2e\n", it + 1,
                  ell, std::sqrt(std::max(0.0, 1.0 - frac * frac)));
        }
        Arena ar(s);
        round_tt<double>(s, ar, r.get(), std::min(1e-2, inner), 0);
      }
      // the correction is noise-like and of higher rank than u: enrich twice as fast
      auto d = default_x0(s, f, QTT_F64);
      auto zd = default_z0(s, f, 2 * rho, QTT_F64);
      OuterCheck oc;
      oc.u = u.get();
      oc.f = f;
      oc.tol = o.tol;
      amen_run<double>(s, K, r.get(), d.get(), zd.get(), inner, o, inf, mixed, true, 0.0, oc);
      // u + d is rounded only at the level of FP64 noise: K amplifies the
      // high-frequency part of a truncation error by up to its condition
      // number (~4^L), so truncating u + d at anything near tol would
      // undo the correction
      u = own(tt_sum<double>(s, 1.0, u.get(), 1.0, d.get()));
      Arena ar(s);
      round_tt<double>(s, ar, u.get(), 1e-14, o.max_rank > 0 ? o.max_rank : 0);
      QTT_CUDA(cudaStreamSynchronize(s));
      inf->refinements += 1;
      inf->refine_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_ref).count();
    }
    *xout = u.release();
  }
  inf->status = rc;
  int mr = 0;
  for (int k = 0; k <= (*xout)->d; ++k) mr = std::max(mr, (*xout)->r[k]);
  inf->max_rank = mr;
  inf->erank = erank_of(*xout);
  return rc;
}

}  // namespace qtt

extern "C" int qtt_autotune_table(int cap, int* count, int* r0_bucket, int* r1_bucket, double* us_tc,
                                  double* us_simt) {
  std::lock_guard<std::mutex> lk(qtt::g_tune_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  int n = 0;
  for (const auto& e : qtt::g_tune) {
    if (e.dev != dev) continue;
    if (n < cap) {
      if (r0_bucket) r0_bucket[n] = e.b0;
      if (r1_bucket) r1_bucket[n] = e.b1;
      if (us_tc) us_tc[n] = e.us_tc;
      if (us_simt) us_simt[n] = e.us_simt;
    }
    ++n;
  }
  if (count) *count = n;
  return QTT_OK;
}

extern "C" int qtt_solve(const qtt_tensor* K, const qtt_tensor* f, const qtt_tensor* x0, const qtt_tensor* z0,
                         const qtt_solve_opts* opts, qtt_tensor** x, qtt_solve_info* info, void* stream) {
  try {
    qtt::StreamScope scope_(reinterpret_cast<cudaStream_t>(stream));
    int rc = qtt::solve(K, f, x0, z0, opts, x, info, reinterpret_cast<cudaStream_t>(stream));
    if (rc == QTT_ENOCONV) qtt::set_last_error("qtt_solve: tolerance not reached");
    return rc;
  } catch (const qtt::QttError& e) {
    qtt::set_last_error(e.what());
    if (info) info->status = e.code;
    return e.code;
  } catch (const std::exception& e) {
    qtt::set_last_error(e.what());
    return QTT_EINVAL;
  }
}
