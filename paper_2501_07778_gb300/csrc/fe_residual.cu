// Full-format FP64 residual f - K u of an assembled problem, with K applied
// as the finite-element operator it represents instead of the QTT product.
//
// The exact QTT route forms K u with ranks R r (about 3 500 - 10 000 at
// L = 12) and expands it: ~1e12 FP64 flops per check on a GPU whose FP64
// pipe runs 1.06 TFLOP/s.  Here u and f are expanded at their own ranks
// (O(N r) flops) into the canonical layout (patch-major, node i + n j, the
// two components interleaved) and the operator is applied node by node:
//   * patch stiffness K^(m): every element of a unit-square patch is the
//     same square, so (K^(m) v)_node is the sum over the (up to four)
//     elements around the node of the 8 x 8 element matrix (Section 3.4,
//     2 x 2 Gauss, plane-stress C) times the element's corner values;
//   * concatenation (Section 3.6, the reading of the assembly): a node held
//     by several patch copies gets, in every copy's row, the sum of all
//     copies' stiffness rows plus gamma (cnt u_a - sum of the copies' u) on
//     both components; copies are grouped by physical node on the host;
//   * masks (Section 3.8): K_bc u = M K (M u) + (I - M) u, a node being
//     constrained in a component in every copy if any copy lies on a side
//     constrained in that component.
// One pass reads u, f and the stencil output once: HBM-bound.  The result
// differs from the QTT product only by the assembly's rounding of K.
#include <algorithm>
#include <cmath>
#include <map>
#include <utility>
#include <vector>

#include "common.cuh"
#include "tt_ops.cuh"

namespace qtt {
namespace {

constexpr unsigned char FE_FIX_X = 1, FE_FIX_Y = 2, FE_SHARED = 4;

struct FeParams {
  int L, q, n;
  double gamma;
  double Ke[64];     // element matrix, row-major, DOFs (ux, uy) of corners 0..3
  int bc[64];        // 4 side flags per patch (q <= 16)
};

// corner c of the element with lower-left node (ei, ej): (ei + CX[c], ej + CY[c])
__constant__ int CX[4] = {0, 1, 1, 0};
__constant__ int CY[4] = {0, 0, 1, 1};

// Element stiffness of an h x h square, plane stress, 2 x 2 Gauss rule
// (exact for the bilinear shape functions), corners counter-clockwise
// from the lower left, DOFs (ux_c, uy_c).
void element_matrix(double E, double nu, double h, double* Ke) {
  const double e = E / (1.0 - nu * nu);
  const double C[3][3] = {{e, e * nu, 0.0}, {e * nu, e, 0.0}, {0.0, 0.0, 0.5 * e * (1.0 - nu)}};
  const double sx[4] = {-1, 1, 1, -1}, sy[4] = {-1, -1, 1, 1};
  const double g = 1.0 / std::sqrt(3.0);
  for (int i = 0; i < 64; ++i) Ke[i] = 0.0;
  for (int gx = 0; gx < 2; ++gx)
    for (int gy = 0; gy < 2; ++gy) {
      const double xi = gx ? g : -g, eta = gy ? g : -g;
      double B[3][8] = {};
      for (int c = 0; c < 4; ++c) {
        const double dx = sx[c] * (1.0 + sy[c] * eta) / 4.0 * (2.0 / h);   // d phi_c / dx
        const double dy = sy[c] * (1.0 + sx[c] * xi) / 4.0 * (2.0 / h);    // d phi_c / dy
        B[0][2 * c] = dx;
        B[1][2 * c + 1] = dy;
        B[2][2 * c] = dy;
        B[2][2 * c + 1] = dx;
      }
      const double w = h * h / 4.0;   // unit Gauss weights times det J
      for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b) {
          double v = 0.0;
          for (int r = 0; r < 3; ++r)
            for (int t = 0; t < 3; ++t) v += B[r][a] * C[r][t] * B[t][b];
          Ke[a * 8 + b] += w * v;
        }
    }
}

__global__ void fe_flags_kernel(FeParams p, unsigned char* flags) {
  const long long nn = (long long)p.n * p.n, total = nn * p.q;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(t / nn);
    const long long node = t % nn;
    const int i = (int)(node % p.n), j = (int)(node / p.n);
    int f = 0;
    if (i == 0) f |= p.bc[4 * m + 0];
    if (i == p.n - 1) f |= p.bc[4 * m + 1];
    if (j == 0) f |= p.bc[4 * m + 2];
    if (j == p.n - 1) f |= p.bc[4 * m + 3];
    flags[t] = (unsigned char)f;
  }
}

// copies of one physical node: every copy takes the union of their flags
__global__ void fe_group_flags_kernel(int ngroups, const int* gstart, const long long* gidx, unsigned char* flags) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroups) return;
  unsigned char u = 0;
  for (int k = gstart[g]; k < gstart[g + 1]; ++k) u |= flags[gidx[k]] & (FE_FIX_X | FE_FIX_Y);
  for (int k = gstart[g]; k < gstart[g + 1]; ++k) flags[gidx[k]] = u | FE_SHARED;
}

// y = K^(m) (M u) for every node of every patch (canonical layout)
__global__ void __launch_bounds__(256) fe_stencil_kernel(FeParams p, const double* __restrict__ u,
                                                         const unsigned char* __restrict__ flags, double* __restrict__ y) {
  __shared__ double Ke[64];
  if (threadIdx.x < 64) Ke[threadIdx.x] = p.Ke[threadIdx.x];
  __syncthreads();
  const int n = p.n;
  const long long nn = (long long)n * n, total = nn * p.q;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long base = (t / nn) * nn;
    const long long node = t % nn;
    const int i = (int)(node % n), j = (int)(node / n);
    double a0 = 0.0, a1 = 0.0;
    // the node is corner `a` of the element with lower-left node (i - CX[a], j - CY[a])
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int ei = i - CX[a], ej = j - CY[a];
      if (ei < 0 || ej < 0 || ei >= n - 1 || ej >= n - 1) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const long long v = base + (ei + CX[b]) + (long long)n * (ej + CY[b]);
        const unsigned char fl = flags[v];
        const double ux = (fl & FE_FIX_X) ? 0.0 : u[2 * v];
        const double uy = (fl & FE_FIX_Y) ? 0.0 : u[2 * v + 1];
        a0 += Ke[(2 * a) * 8 + 2 * b] * ux + Ke[(2 * a) * 8 + 2 * b + 1] * uy;
        a1 += Ke[(2 * a + 1) * 8 + 2 * b] * ux + Ke[(2 * a + 1) * 8 + 2 * b + 1] * uy;
      }
    }
    y[2 * t] = a0;
    y[2 * t + 1] = a1;
  }
}

__device__ double fe_block_sum(double v, double* red) {
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
  return r;
}

// sum of (f - K_bc u)^2 over nodes held by one copy, and of f^2 over all
__global__ void __launch_bounds__(256) fe_residual_kernel(long long total, const double* __restrict__ u,
                                                          const double* __restrict__ f,
                                                          const unsigned char* __restrict__ flags,
                                                          const double* __restrict__ y, double* acc,
                                                          double* __restrict__ rvec) {
  __shared__ double red[32];
  double r2 = 0.0, f2 = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const unsigned char fl = flags[t];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double fv = f[2 * t + c];
      f2 += fv * fv;
      if (fl & FE_SHARED) continue;
      const double ku = (fl & (1 << c)) ? u[2 * t + c] : y[2 * t + c];
      const double r = fv - ku;
      r2 += r * r;
      if (rvec) rvec[2 * t + c] = r;
    }
  }
  r2 = fe_block_sum(r2, red);
  f2 = fe_block_sum(f2, red);
  if (threadIdx.x == 0) {
    atomicAdd(&acc[0], r2);
    atomicAdd(&acc[1], f2);
  }
}

// the rows of shared nodes: summed stiffness rows plus the gamma coupling
__global__ void fe_group_residual_kernel(double gamma, int ngroups, const int* gstart, const long long* gidx,
                                         const double* __restrict__ u, const double* __restrict__ f,
                                         const unsigned char* __restrict__ flags, const double* __restrict__ y,
                                         double* acc, double* __restrict__ rvec) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0;
  if (g < ngroups) {
    const int k0 = gstart[g], k1 = gstart[g + 1];
    const double cnt = (double)(k1 - k0);
    const unsigned char fl = flags[gidx[k0]];
    for (int c = 0; c < 2; ++c) {
      const bool fixed = (fl & (1 << c)) != 0;
      double sy = 0.0, su = 0.0;
      for (int k = k0; k < k1; ++k) {
        sy += y[2 * gidx[k] + c];
        su += fixed ? 0.0 : u[2 * gidx[k] + c];
      }
      for (int k = k0; k < k1; ++k) {
        const long long v = gidx[k];
        const double uv = u[2 * v + c];
        const double row = fixed ? uv : sy + gamma * (cnt * uv - su);
        const double r = f[2 * v + c] - row;
        r2 += r * r;
        if (rvec) rvec[2 * v + c] = r;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  if ((threadIdx.x & 31) == 0 && r2 != 0.0) atomicAdd(&acc[0], r2);
}

// y = K_bc x at nodes held by one copy (y holds the stencil output)
__global__ void fe_rows_kernel(long long total, const double* __restrict__ x, const unsigned char* __restrict__ flags,
                               double* __restrict__ y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const unsigned char fl = flags[t];
    if (fl & FE_SHARED) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (fl & (1 << c)) y[2 * t + c] = x[2 * t + c];
  }
}

// y = K_bc x at shared nodes: summed stiffness rows plus gamma coupling
// (one thread per group; reads the stencil rows ys, writes y)
__global__ void fe_group_rows_kernel(double gamma, int ngroups, const int* gstart, const long long* gidx,
                                     const double* __restrict__ x, const unsigned char* __restrict__ flags,
                                     const double* __restrict__ ys, double* __restrict__ y) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroups) return;
  const int k0 = gstart[g], k1 = gstart[g + 1];
  const double cnt = (double)(k1 - k0);
  const unsigned char fl = flags[gidx[k0]];
  for (int c = 0; c < 2; ++c) {
    const bool fixed = (fl & (1 << c)) != 0;
    double sy = 0.0, su = 0.0;
    for (int k = k0; k < k1; ++k) {
      sy += ys[2 * gidx[k] + c];
      su += fixed ? 0.0 : x[2 * gidx[k] + c];
    }
    for (int k = k0; k < k1; ++k) {
      const long long v = gidx[k];
      y[2 * v + c] = fixed ? x[2 * v + c] : sy + gamma * (cnt * x[2 * v + c] - su);
    }
  }
}

// Copies of physical nodes shared by two or more patches, as index lists
// into the canonical node array (m n^2 + i + n j).  Patches are unit squares
// at integer offsets, so only patch-boundary nodes can coincide.
void shared_groups(const FeOperator& op, std::vector<int>& start, std::vector<long long>& idx) {
  const int n = 1 << op.L;
  const long long nn = (long long)n * n;
  std::map<std::pair<long long, long long>, std::vector<long long>> where;
  for (int m = 0; m < op.q; ++m) {
    const long long ox = (long long)op.patch_xy[2 * m] * (n - 1), oy = (long long)op.patch_xy[2 * m + 1] * (n - 1);
    for (int t = 0; t < 4 * (n - 1); ++t) {
      int i, j;   // walk the boundary once
      if (t < n - 1) { i = t; j = 0; }
      else if (t < 2 * (n - 1)) { i = n - 1; j = t - (n - 1); }
      else if (t < 3 * (n - 1)) { i = n - 1 - (t - 2 * (n - 1)); j = n - 1; }
      else { i = 0; j = n - 1 - (t - 3 * (n - 1)); }
      where[{ox + i, oy + j}].push_back(m * nn + i + (long long)n * j);
    }
  }
  start.assign(1, 0);
  idx.clear();
  for (auto& kv : where) {
    if (kv.second.size() < 2) continue;
    for (long long v : kv.second) idx.push_back(v);
    start.push_back((int)idx.size());
  }
}

}  // namespace

bool has_fe_operator(const qtt_tensor* K) { return K && K->fe && K->prec == QTT_F64; }

// y = K_bc x for full canonical vectors x, y (device, 2 q n^2 doubles each)
void fe_apply(cudaStream_t s, const qtt_tensor* K, const double* x, double* y) {
  QTT_REQUIRE(has_fe_operator(K), "fe_apply: K does not come from qtt_assemble_stiffness");
  const FeOperator& op = *K->fe;
  const int n = 1 << op.L;
  const long long nn = (long long)n * n, total = nn * op.q;
  FeParams p{};
  p.L = op.L;
  p.q = op.q;
  p.n = n;
  p.gamma = op.gamma;
  element_matrix(op.E, op.nu, 1.0 / (n - 1.0), p.Ke);
  for (int i = 0; i < 4 * op.q; ++i) p.bc[i] = op.bc[i];
  Arena ar(s);
  unsigned char* flags = ar.alloc<unsigned char>(total);
  fe_flags_kernel<<<grid_for_n(total, 8), 256, 0, s>>>(p, flags);
  QTT_CHECK_LAUNCH();
  std::vector<int> gstart;
  std::vector<long long> gidx;
  shared_groups(op, gstart, gidx);
  const int ngroups = (int)gstart.size() - 1;
  int* d_start = nullptr;
  long long* d_idx = nullptr;
  if (ngroups > 0) {
    d_start = ar.alloc<int>(gstart.size());
    d_idx = ar.alloc<long long>(gidx.size());
    QTT_CUDA(cudaMemcpyAsync(d_start, gstart.data(), sizeof(int) * gstart.size(), cudaMemcpyHostToDevice, s));
    QTT_CUDA(cudaMemcpyAsync(d_idx, gidx.data(), sizeof(long long) * gidx.size(), cudaMemcpyHostToDevice, s));
    fe_group_flags_kernel<<<(ngroups + 127) / 128, 128, 0, s>>>(ngroups, d_start, d_idx, flags);
    QTT_CHECK_LAUNCH();
  }
  double* ys = ngroups > 0 ? ar.alloc<double>(2 * total) : y;   // stencil rows
  fe_stencil_kernel<<<grid_for_n(total, 8), 256, 0, s>>>(p, x, flags, ys);
  QTT_CHECK_LAUNCH();
  if (ngroups > 0) {
    QTT_CUDA(cudaMemcpyAsync(y, ys, sizeof(double) * 2 * total, cudaMemcpyDeviceToDevice, s));
    fe_group_rows_kernel<<<(ngroups + 127) / 128, 128, 0, s>>>(op.gamma, ngroups, d_start, d_idx, x, flags, ys, y);
    QTT_CHECK_LAUNCH();
  }
  fe_rows_kernel<<<grid_for_n(total, 8), 256, 0, s>>>(total, x, flags, y);
  QTT_CHECK_LAUNCH();
}

namespace {
// ||f - K (u + u2)|| / ||f|| (u2 may be NULL) with K applied as the
// assembled finite-element operator; rvec (NULL, or 2 q 4^L doubles on the
// device) receives the residual vector in canonical order
double residual_fe_impl(cudaStream_t s, Arena& ar, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* u2,
                        const qtt_tensor* f, double* rvec) {
  QTT_REQUIRE(has_fe_operator(K), "residual: K does not come from qtt_assemble_stiffness");
  const FeOperator& op = *K->fe;
  QTT_REQUIRE(op.q >= 1 && op.q <= 16, "residual: patch count out of range");
  QTT_REQUIRE(u->prec == QTT_F64 && f->prec == QTT_F64 && (!u2 || u2->prec == QTT_F64),
              "residual: u and f must be FP64");
  const int n = 1 << op.L;
  const long long nn = (long long)n * n, total = nn * op.q;
  FeParams p{};
  p.L = op.L;
  p.q = op.q;
  p.n = n;
  p.gamma = op.gamma;
  element_matrix(op.E, op.nu, 1.0 / (n - 1.0), p.Ke);
  for (int i = 0; i < 4 * op.q; ++i) p.bc[i] = op.bc[i];
  double* uf = ar.alloc<double>(2 * total);
  double* ff = ar.alloc<double>(2 * total);
  double* y = ar.alloc<double>(2 * total);
  unsigned char* flags = ar.alloc<unsigned char>(total);
  double* acc = ar.alloc<double>(2);
  to_full<double>(s, ar, u, uf, (size_t)(2 * total), QTT_ORDER_CANONICAL);
  if (u2) {   // the sum's expansion: y serves as scratch before the stencil
    to_full<double>(s, ar, u2, y, (size_t)(2 * total), QTT_ORDER_CANONICAL);
    axpby<double>(s, (size_t)(2 * total), 1.0, y, 1.0, uf);
  }
  to_full<double>(s, ar, f, ff, (size_t)(2 * total), QTT_ORDER_CANONICAL);
  fe_flags_kernel<<<grid_for_n(total, 8), 256, 0, s>>>(p, flags);
  QTT_CHECK_LAUNCH();
  std::vector<int> gstart;
  std::vector<long long> gidx;
  shared_groups(op, gstart, gidx);
  const int ngroups = (int)gstart.size() - 1;
  int* d_start = nullptr;
  long long* d_idx = nullptr;
  if (ngroups > 0) {
    d_start = ar.alloc<int>(gstart.size());
    d_idx = ar.alloc<long long>(gidx.size());
    QTT_CUDA(cudaMemcpyAsync(d_start, gstart.data(), sizeof(int) * gstart.size(), cudaMemcpyHostToDevice, s));
    QTT_CUDA(cudaMemcpyAsync(d_idx, gidx.data(), sizeof(long long) * gidx.size(), cudaMemcpyHostToDevice, s));
    fe_group_flags_kernel<<<(ngroups + 127) / 128, 128, 0, s>>>(ngroups, d_start, d_idx, flags);
    QTT_CHECK_LAUNCH();
  }
  fe_stencil_kernel<<<grid_for_n(total, 8), 256, 0, s>>>(p, uf, flags, y);
  QTT_CHECK_LAUNCH();
  QTT_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(double), s));
  fe_residual_kernel<<<grid_for_n(total, 4), 256, 0, s>>>(total, uf, ff, flags, y, acc, rvec);
  QTT_CHECK_LAUNCH();
  if (ngroups > 0) {
    fe_group_residual_kernel<<<(ngroups + 127) / 128, 128, 0, s>>>(op.gamma, ngroups, d_start, d_idx, uf, ff, flags,
                                                                   y, acc, rvec);
    QTT_CHECK_LAUNCH();
  }
  double h[2] = {0.0, 0.0};
  QTT_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  QTT_CUDA(cudaStreamSynchronize(s));
  return h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
}
}  // namespace

double residual_fe(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* u2,
                   const qtt_tensor* f) {
  Arena ar(s);
  return residual_fe_impl(s, ar, K, u, u2, f, nullptr);
}

// f - K u formed element by element in FP64 (the assembled operator, as in
// residual_fe), reordered to QTT order and compressed by TT-SVD at relative
// accuracy eps with ranks <= max_rank; *rel = ||f - K u|| / ||f||.
qtt_tensor* residual_fe_tt(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f, double eps,
                           int max_rank, double* rel) {
  QTT_REQUIRE(has_fe_operator(K), "residual: K does not come from qtt_assemble_stiffness");
  const FeOperator& op = *K->fe;
  const long long total = 2LL * op.q << (2 * op.L);
  Arena ar(s);
  double* rc = ar.alloc<double>(total);
  const double r = residual_fe_impl(s, ar, K, u, nullptr, f, rc);
  if (rel) *rel = r;
  double* rz = ar.alloc<double>(total);
  from_canonical<double>(s, rc, rz, op.L, op.q);
  return tt_svd_full(s, ar, rz, f->d, f->n, eps, max_rank);
}

}  // namespace qtt

extern "C" int qtt_fe_apply(const qtt_tensor* K, const void* x, void* y, size_t n_elems, void* stream) {
  try {
    QTT_REQUIRE(K && x && y, "qtt_fe_apply: null argument");
    QTT_REQUIRE(qtt::has_fe_operator(K), "qtt_fe_apply: K does not come from qtt_assemble_stiffness");
    const long long nn = 1LL << (2 * K->fe->L);
    QTT_REQUIRE((long long)n_elems == 2 * K->fe->q * nn, "qtt_fe_apply: n_elems must be 2 q 4^L");
    QTT_REQUIRE(x != y, "qtt_fe_apply: x and y must not alias");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    qtt::StreamScope scope_(s);
    qtt::fe_apply(s, K, static_cast<const double*>(x), static_cast<double*>(y));
    return QTT_OK;
  } catch (const qtt::QttError& e) {
    qtt::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    qtt::set_last_error(e.what());
    return QTT_EINVAL;
  }
}

extern "C" int qtt_residual_fe(const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f, double* out,
                               void* stream) {
  try {
    QTT_REQUIRE(K && u && f && out, "qtt_residual_fe: null argument");
    QTT_REQUIRE(K->is_matrix && !u->is_matrix && !f->is_matrix && K->d == u->d && K->d == f->d,
                "qtt_residual_fe: K must be an MPO and u, f MPS of equal length");
    for (int k = 0; k < K->d; ++k)
      QTT_REQUIRE(K->n[k] == u->n[k] && K->n[k] == f->n[k], "qtt_residual_fe: mode sizes differ");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    qtt::StreamScope scope_(s);
    *out = qtt::residual_fe(s, K, u, nullptr, f);
    return QTT_OK;
  } catch (const qtt::QttError& e) {
    qtt::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    qtt::set_last_error(e.what());
    return QTT_EINVAL;
  }
}

extern "C" int qtt_residual_fe_tt(const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f, double eps,
                                  int max_rank, qtt_tensor** r, double* rel, void* stream) {
  try {
    QTT_REQUIRE(K && u && f && r, "qtt_residual_fe_tt: null argument");
    QTT_REQUIRE(K->is_matrix && !u->is_matrix && !f->is_matrix && K->d == u->d && K->d == f->d,
                "qtt_residual_fe_tt: K must be an MPO and u, f MPS of equal length");
    for (int k = 0; k < K->d; ++k)
      QTT_REQUIRE(K->n[k] == u->n[k] && K->n[k] == f->n[k], "qtt_residual_fe_tt: mode sizes differ");
    QTT_REQUIRE(eps >= 1e-6 && eps < 1.0, "qtt_residual_fe_tt: eps must lie in [1e-6, 1)");
    QTT_REQUIRE(max_rank >= 1, "qtt_residual_fe_tt: max_rank must be positive");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    qtt::StreamScope scope_(s);
    *r = qtt::residual_fe_tt(s, K, u, f, eps, max_rank, rel);
    return QTT_OK;
  } catch (const qtt::QttError& e) {
    qtt::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    qtt::set_last_error(e.what());
    return QTT_EINVAL;
  }
}
