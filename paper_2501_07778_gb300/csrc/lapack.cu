// Dense factorizations written from the textbook mathematics:
//  * Householder QR in compact WY form (Golub & Van Loan, Sec. 5.1-5.2):
//    single-CTA panel factorisation of 32 columns, trailing update and the
//    explicit Q by three GEMMs per panel;
//  * one-sided (Hestenes) Jacobi SVD of the triangular factor with the
//    round-robin parallel ordering (Demmel & Veselic 1992);
//  * LU with partial pivoting: single-CTA panel, triangular solve of the
//    block row and GEMM trailing update; blocked triangular solves.
#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>

#include "common.cuh"

namespace qtt {
namespace {

constexpr int NB = 16;         // panel width (a panel runs on one SM: its N nb^2 FP64 work grows with nb)
constexpr size_t kJacobiSmem = 200 * 1024;   // dynamic shared memory of the in-smem Jacobi sweeps
constexpr int PT = 1024;       // panel kernel threads

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ double block_sum(double v, double* red) {
  v = wsum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
    r = wsum(r);
    if (l == 0) red[32] = r;
  }
  __syncthreads();
  return red[32];
}

// Householder panel: A is the m x jb panel (lda), V receives the reflectors
// (m x jb, ld ldv, unit diagonal, zeros above), Tm the jb x jb upper
// triangular factor (ld NB) with H_1..H_jb = I - V Tm V^T.
template <typename T>
__global__ void __launch_bounds__(PT) qr_panel_kernel(int m, int jb, T* A, int lda, T* V, int ldv, T* Tm) {
  __shared__ double red[33];
  __shared__ double s_tau, s_scale, s_beta;
  __shared__ double y[NB];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int c = 0; c < jb; ++c) {
    T* a = A + (long long)c * lda;
    double part = 0.0;
    for (int i = c + 1 + tid; i < m; i += PT) part += (double)a[i] * (double)a[i];
    double sigma = block_sum<T>(part, red);
    if (tid == 0) {
      double alpha = (c < m) ? (double)a[c] : 0.0;
      double tau = 0.0, scale = 0.0, beta = alpha;
      if (sigma > 0.0) {
        double nrm = sqrt(alpha * alpha + sigma);
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      s_tau = tau;
      s_scale = scale;
      s_beta = beta;
    }
    __syncthreads();
    const double tau = s_tau, scale = s_scale;
    T* v = V + (long long)c * ldv;
    for (int i = tid; i < m; i += PT) {
      if (i < c) v[i] = T(0);
      else if (i == c) v[i] = T(1);
      else {
        T vi = (T)((double)a[i] * scale);
        v[i] = vi;
        a[i] = vi;
      }
    }
    if (tid == 0 && c < m) a[c] = (T)s_beta;
    __syncthreads();
    // apply H_c to the remaining panel columns (one warp per column)
    for (int j = c + 1 + warp; j < jb; j += PT / 32) {
      T* aj = A + (long long)j * lda;
      double d = 0.0;
      for (int i = c + lane; i < m; i += 32) d += (double)v[i] * (double)aj[i];
      d = wsum(d) * tau;
      for (int i = c + lane; i < m; i += 32) aj[i] = (T)((double)aj[i] - d * (double)v[i]);
    }
    // T column: T[0:c, c] = -tau T[0:c, 0:c] (V[:, 0:c]^T v_c), T[c, c] = tau
    for (int w = warp; w < c; w += PT / 32) {
      const T* vw = V + (long long)w * ldv;
      double d = 0.0;
      for (int i = c + lane; i < m; i += 32) d += (double)vw[i] * (double)v[i];
      d = wsum(d);
      if (lane == 0) y[w] = d;
    }
    __syncthreads();
    if (tid < c) {
      double acc = 0.0;
      for (int s2 = tid; s2 < c; ++s2) acc += (double)Tm[tid + s2 * NB] * y[s2];
      Tm[tid + c * NB] = (T)(-tau * acc);
    }
    if (tid == 0) Tm[c + c * NB] = (T)tau;
    for (int t = tid; t < NB; t += PT)
      if (t > c) Tm[t + c * NB] = T(0);
    __syncthreads();
  }
}

template <typename T>
__global__ void set_identity_kernel(T* Q, int m, int k, int ldq) {
  long long total = (long long)m * k;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % m), j = (int)(t / m);
    Q[i + (long long)j * ldq] = (i == j) ? T(1) : T(0);
  }
}

template <typename T>
__global__ void upper_copy_kernel(const T* A, int lda, T* R, int ldr, int k, int n) {
  long long total = (long long)k * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % k), j = (int)(t / k);
    R[i + (long long)j * ldr] = (i <= j) ? A[i + (long long)j * lda] : T(0);
  }
}

inline int grid_for(long long n) { return grid_for_n(n, 16); }

// ---------------------------------------------------------------------------
// One-sided Jacobi on W (m x n, ldw) accumulating V (n x n, ldv); single CTA.
// ---------------------------------------------------------------------------
template <typename T, typename Acc>
__device__ int jacobi_body(int m, int n, T* W, int ldw, T* Vm, int ldv, int max_sweeps, int* rotated_flag);

template <typename T, typename Acc = double>
__global__ void __launch_bounds__(1024) jacobi_kernel(int m, int n, T* W, int ldw, T* Vm, int ldv, int max_sweeps,
                                                      int* sweeps_out) {
  __shared__ int rotated;
  const int sweep = jacobi_body<T, Acc>(m, n, W, ldw, Vm, ldv, max_sweeps, &rotated);
  if (threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
}

// The same sweeps with W (and V when both fit) held in shared memory for the
// whole factorisation: every round reads and rewrites two columns of each
// pair, which from global memory costs an L2 round trip per access.
template <typename T, typename Acc = double>
__global__ void __launch_bounds__(1024) jacobi_smem_kernel(int m, int n, T* W, int ldw, T* Vm, int ldv, int max_sweeps,
                                                           int v_in_smem) {
  extern __shared__ __align__(16) unsigned char jsm[];
  __shared__ int rotated;
  T* Ws = reinterpret_cast<T*>(jsm);
  T* Vs = v_in_smem ? Ws + (size_t)m * n : Vm;
  const int ldvs = v_in_smem ? n : ldv;
  for (long long t = threadIdx.x; t < (long long)m * n; t += blockDim.x) Ws[t] = W[(t % m) + (t / m) * (long long)ldw];
  if (v_in_smem)
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) Vs[t] = Vm[(t % n) + (t / n) * (long long)ldv];
  __syncthreads();
  jacobi_body<T, Acc>(m, n, Ws, m, Vs, ldvs, max_sweeps, &rotated);
  __syncthreads();
  for (long long t = threadIdx.x; t < (long long)m * n; t += blockDim.x) W[(t % m) + (t / m) * (long long)ldw] = Ws[t];
  if (v_in_smem)
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) Vm[(t % n) + (t / n) * (long long)ldv] = Vs[t];
}

template <typename T, typename Acc>
__device__ int jacobi_body(int m, int n, T* W, int ldw, T* Vm, int ldv, int max_sweeps, int* rotated_flag) {
  int& rotated = *rotated_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int np = n + (n & 1);                  // even number of positions
  const Acc tol = (Acc)(1e-15 * (double)(m > 1 ? m : 1));
  const Acc tolf = (sizeof(T) == 4) ? (Acc)(1e-7 * (double)(m > 1 ? m : 1)) : tol;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int pi = warp; pi < np / 2; pi += nw) {
        // pair number pi of round `round` in the round-robin tournament
        int p, q;
        if (pi == 0) {
          p = round % (np - 1);
          q = np - 1;
        } else {
          p = (round + pi) % (np - 1);
          q = (round - pi + (np - 1)) % (np - 1);
        }
        if (p > q) { int t = p; p = q; q = t; }
        if (q >= n) continue;                  // dummy position for odd n
        T* wp = W + (long long)p * ldw;
        T* wq = W + (long long)q * ldw;
        Acc al = 0, be = 0, ga = 0;
        for (int i = lane; i < m; i += 32) {
          Acc a = wp[i], b = wq[i];
          al += a * a;
          be += b * b;
          ga += a * b;
        }
        al = wsum(al);
        be = wsum(be);
        ga = wsum(ga);
        if (ga == (Acc)0 || !(fabs(ga) > tolf * sqrt(al * be))) continue;
        Acc zeta = (be - al) / ((Acc)2 * ga);
        Acc t = (zeta >= (Acc)0 ? (Acc)1 : (Acc)-1) / (fabs(zeta) + sqrt((Acc)1 + zeta * zeta));
        Acc cs = (Acc)1 / sqrt((Acc)1 + t * t), sn = cs * t;
        for (int i = lane; i < m; i += 32) {
          Acc a = wp[i], b = wq[i];
          wp[i] = (T)(cs * a - sn * b);
          wq[i] = (T)(sn * a + cs * b);
        }
        T* vp = Vm + (long long)p * ldv;
        T* vq = Vm + (long long)q * ldv;
        for (int i = lane; i < n; i += 32) {
          Acc a = vp[i], b = vq[i];
          vp[i] = (T)(cs * a - sn * b);
          vq[i] = (T)(sn * a + cs * b);
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  return sweep;
}

// ---------------------------------------------------------------------------
// The same one-sided Jacobi sweeps on many SMs: the np/2 pairs of a round go
// to the warps of the whole grid (one pair per warp, one warp per CTA while
// the pairs fit the SMs), so the FP64 dot products and rotations of a round
// run on up to np/2 SMs instead of one; a grid barrier separates the rounds.
// Column data written in one round is read by other SMs in the next, so the
// loads bypass L1 (__ldcg).  rot[s] counts the warps that rotated in sweep s
// (zeroed by the host) and rot[max_sweeps + s] the warps with a rotation
// above the quadratic-convergence threshold; every thread reads them after
// the sweep's last barrier, so all CTAs take the same stop decision.
// Cooperative launch only.
// ---------------------------------------------------------------------------
template <typename T, typename Acc>
__global__ void jacobi_coop_kernel(int m, int n, T* W, int ldw, T* Vm, int ldv, int max_sweeps, unsigned* rot,
                                   int* sweeps_out) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
  const int nwarps = gridDim.x * wpb;
  const int np = n + (n & 1);
  const Acc tol = (Acc)(1e-15 * (double)(m > 1 ? m : 1));
  const Acc tolf = (sizeof(T) == 4) ? (Acc)(1e-7 * (double)(m > 1 ? m : 1)) : tol;
  int sweep = 0;
  // a sweep whose rotations are all tiny (relative off-diagonal below
  // 1e-8 in FP64) leaves the columns orthogonal to working accuracy
  // (quadratic convergence), so it ends the sweeps without a confirming one
  const Acc big = (sizeof(T) == 8) ? (Acc)1e-8 : (Acc)1e-4;
  constexpr int JT = 8;                       // register path: columns of <= 256 rows
  const bool inreg = m <= 32 * JT && n <= 32 * JT;
  for (; sweep < max_sweeps; ++sweep) {
    bool any = false, large = false;
    for (int round = 0; round < np - 1; ++round) {
      for (int pi = gw; pi < np / 2; pi += nwarps) {
        int p, q;
        if (pi == 0) {
          p = round % (np - 1);
          q = np - 1;
        } else {
          p = (round + pi) % (np - 1);
          q = (round - pi + (np - 1)) % (np - 1);
        }
        if (p > q) { int t = p; p = q; q = t; }
        if (q >= n) continue;
        T* wp = W + (long long)p * ldw;
        T* wq = W + (long long)q * ldw;
        T* vp = Vm + (long long)p * ldv;
        T* vq = Vm + (long long)q * ldv;
        Acc al = 0, be = 0, ga = 0;
        if (inreg) {
          // the pair's four columns in registers: every load of the round
          // is issued at once, and the rotation reuses the loaded values
          Acc a[JT], b[JT], va[JT], vb[JT];
#pragma unroll
          for (int t = 0; t < JT; ++t) {
            const int i = lane + 32 * t;
            a[t] = i < m ? (Acc)__ldcg(wp + i) : (Acc)0;
            b[t] = i < m ? (Acc)__ldcg(wq + i) : (Acc)0;
            va[t] = i < n ? (Acc)__ldcg(vp + i) : (Acc)0;
            vb[t] = i < n ? (Acc)__ldcg(vq + i) : (Acc)0;
          }
#pragma unroll
          for (int t = 0; t < JT; ++t) {
            al += a[t] * a[t];
            be += b[t] * b[t];
            ga += a[t] * b[t];
          }
          al = wsum(al);
          be = wsum(be);
          ga = wsum(ga);
          if (ga == (Acc)0 || !(fabs(ga) > tolf * sqrt(al * be))) continue;
          if (fabs(ga) > big * sqrt(al * be)) large = true;
          Acc zeta = (be - al) / ((Acc)2 * ga);
          Acc t = (zeta >= (Acc)0 ? (Acc)1 : (Acc)-1) / (fabs(zeta) + sqrt((Acc)1 + zeta * zeta));
          Acc cs = (Acc)1 / sqrt((Acc)1 + t * t), sn = cs * t;
#pragma unroll
          for (int u = 0; u < JT; ++u) {
            const int i = lane + 32 * u;
            if (i < m) {
              wp[i] = (T)(cs * a[u] - sn * b[u]);
              wq[i] = (T)(sn * a[u] + cs * b[u]);
            }
            if (i < n) {
              vp[i] = (T)(cs * va[u] - sn * vb[u]);
              vq[i] = (T)(sn * va[u] + cs * vb[u]);
            }
          }
          any = true;
          continue;
        }
        for (int i = lane; i < m; i += 32) {
          Acc a = __ldcg(wp + i), b = __ldcg(wq + i);
          al += a * a;
          be += b * b;
          ga += a * b;
        }
        al = wsum(al);
        be = wsum(be);
        ga = wsum(ga);
        if (ga == (Acc)0 || !(fabs(ga) > tolf * sqrt(al * be))) continue;
        if (fabs(ga) > big * sqrt(al * be)) large = true;
        Acc zeta = (be - al) / ((Acc)2 * ga);
        Acc t = (zeta >= (Acc)0 ? (Acc)1 : (Acc)-1) / (fabs(zeta) + sqrt((Acc)1 + zeta * zeta));
        Acc cs = (Acc)1 / sqrt((Acc)1 + t * t), sn = cs * t;
        for (int i = lane; i < m; i += 32) {
          Acc a = __ldcg(wp + i), b = __ldcg(wq + i);
          wp[i] = (T)(cs * a - sn * b);
          wq[i] = (T)(sn * a + cs * b);
        }
        for (int i = lane; i < n; i += 32) {
          Acc a = __ldcg(vp + i), b = __ldcg(vq + i);
          vp[i] = (T)(cs * a - sn * b);
          vq[i] = (T)(sn * a + cs * b);
        }
        any = true;
      }
      grid.sync();
    }
    if (any && lane == 0) atomicAdd(&rot[sweep], 1u);
    if (large && lane == 0) atomicAdd(&rot[max_sweeps + sweep], 1u);
    grid.sync();
    if (*(volatile unsigned*)&rot[sweep] == 0u) break;
    if (*(volatile unsigned*)&rot[max_sweeps + sweep] == 0u) {
      ++sweep;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && sweeps_out) *sweeps_out = sweep;
}

// column norms -> S, normalise W columns, then sort descending (order[])
template <typename T>
__global__ void __launch_bounds__(1024) svd_finish_kernel(int m, int n, T* W, int ldw, T* S, int* order) {
  extern __shared__ double sh[];
  double* sv = sh;                       // n values
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < n; j += nw) {
    T* w = W + (long long)j * ldw;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s += (double)w[i] * (double)w[i];
    s = sqrt(wsum(s));
    if (lane == 0) sv[j] = s;
    if (s > 0.0)
      for (int i = lane; i < m; i += 32) w[i] = (T)((double)w[i] / s);
  }
  __syncthreads();
  // rank of each value (descending, ties by index) -> position
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    int rank = 0;
    double v = sv[j];
    for (int t = 0; t < n; ++t) {
      double u = sv[t];
      if (u > v || (u == v && t < j)) ++rank;
    }
    order[rank] = j;
    S[rank] = (T)v;
  }
}

template <typename T>
__global__ void gather_cols_kernel(const T* src, int lds, T* dst, int ldd, int rows, int ncols, const int* order,
                                   bool transpose_out) {
  long long total = (long long)rows * ncols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % rows), j = (int)(t / rows);
    T v = src[i + (long long)order[j] * lds];
    if (transpose_out) dst[j + (long long)i * ldd] = v;
    else dst[i + (long long)j * ldd] = v;
  }
}

// ---------------------------------------------------------------------------
// LU panel with partial pivoting: factor columns [j0, j0 + jb) of the full
// n x n matrix A, swapping whole rows of A and of B (nrhs columns).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(PT) lu_panel_kernel(int n, int j0, int jb, T* A, int lda, T* B, int ldb, int nrhs,
                                                      int* info) {
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int s_piv;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int c = j0; c < j0 + jb; ++c) {
    T* col = A + (long long)c * lda;
    double best = -1.0;
    int bi = c;
    for (int i = c + tid; i < n; i += PT) {
      double v = fabs((double)col[i]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int p = c;
      for (int w = 0; w < PT / 32; ++w)
        if (rv[w] > b || (rv[w] == b && ri[w] < p)) { b = rv[w]; p = ri[w]; }
      s_piv = p;
      if (b == 0.0 && info) atomicExch(info, c + 1);
    }
    __syncthreads();
    const int p = s_piv;
    if (p != c) {
      for (int j = tid; j < n; j += PT) {
        T t = A[c + (long long)j * lda];
        A[c + (long long)j * lda] = A[p + (long long)j * lda];
        A[p + (long long)j * lda] = t;
      }
      for (int j = tid; j < nrhs; j += PT) {
        T t = B[c + (long long)j * ldb];
        B[c + (long long)j * ldb] = B[p + (long long)j * ldb];
        B[p + (long long)j * ldb] = t;
      }
    }
    __syncthreads();
    const double piv = (double)col[c];
    const double inv = piv != 0.0 ? 1.0 / piv : 0.0;
    for (int i = c + 1 + tid; i < n; i += PT) col[i] = (T)((double)col[i] * inv);
    __syncthreads();
    // rank-1 update of the rest of the panel (one warp per column)
    for (int j = c + 1 + warp; j < j0 + jb; j += PT / 32) {
      T* aj = A + (long long)j * lda;
      const double u = (double)aj[c];
      for (int i = c + 1 + lane; i < n; i += 32) aj[i] = (T)((double)aj[i] - (double)col[i] * u);
    }
    __syncthreads();
  }
}

// U12 = L11^{-1} A12 for a unit lower jb x jb block: one thread per column
template <typename T>
__global__ void trsm_lower_unit_kernel(int jb, const T* L, int ldl, T* X, int ldx, int ncols) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  T* x = X + (long long)j * ldx;
  for (int i = 0; i < jb; ++i) {
    double v = (double)x[i];
    for (int k = 0; k < i; ++k) v -= (double)L[i + (long long)k * ldl] * (double)x[k];
    x[i] = (T)v;
  }
}

// solve a small triangular block in place (one thread per rhs column)
template <typename T>
__global__ void trsv_block_kernel(int nb, const T* A, int lda, T* X, int ldx, int ncols, bool upper) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncols) return;
  T* x = X + (long long)j * ldx;
  if (!upper) {
    for (int i = 0; i < nb; ++i) {
      double v = (double)x[i];
      for (int k = 0; k < i; ++k) v -= (double)A[i + (long long)k * lda] * (double)x[k];
      x[i] = (T)v;
    }
  } else {
    for (int i = nb - 1; i >= 0; --i) {
      double v = (double)x[i];
      for (int k = i + 1; k < nb; ++k) v -= (double)A[i + (long long)k * lda] * (double)x[k];
      double d = (double)A[i + (long long)i * lda];
      x[i] = (T)(d != 0.0 ? v / d : 0.0);
    }
  }
}

}  // namespace

// FP64 (or FP32) one-sided Jacobi sweeps on W (m x n) accumulating V: the
// cooperative many-SM kernel when the device supports cooperative launch
// and there are enough pairs to spread, else the single-CTA kernel.
template <typename T, typename Acc>
void jacobi_sweeps(cudaStream_t s, Arena& ar, int m, int n, T* W, int ldw, T* Vm, int ldv, int max_sweeps) {
  static int coop = -1;
  if (coop < 0) {
    int dev = 0, v = 0;
    coop = (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && v) ? 1 : 0;
    cudaGetLastError();
  }
  const int pairs = (n + (n & 1)) / 2;
  if (!coop || pairs < 8) {
    jacobi_kernel<T, Acc><<<1, 1024, 0, s>>>(m, n, W, ldw, Vm, ldv, max_sweeps, nullptr);
    QTT_CHECK_LAUNCH();
    return;
  }
  // one warp per pair; one warp per CTA while the pairs fit the SMs
  const int sms = num_sms();
  const int wpb = std::min(8, (pairs + sms - 1) / sms);
  int occ = 0;
  QTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_coop_kernel<T, Acc>, 32 * wpb, 0));
  const int grid = std::max(1, std::min((pairs + wpb - 1) / wpb, sms * std::max(1, occ)));
  unsigned* rot = ar.alloc<unsigned>(2 * max_sweeps);   // rotations, large rotations per sweep
  QTT_CUDA(cudaMemsetAsync(rot, 0, sizeof(unsigned) * 2 * max_sweeps, s));
  int* none = nullptr;
  void* args[] = {&m, &n, &W, &ldw, &Vm, &ldv, &max_sweeps, &rot, &none};
  QTT_CUDA(cudaLaunchCooperativeKernel((void*)jacobi_coop_kernel<T, Acc>, grid, 32 * wpb, args, 0, s));
  count_launch();
}

template <typename T>
void qr(cudaStream_t s, Arena& ar, int m, int n, T* A, int lda, T* Q, int ldq, T* R, int ldr) {
  QTT_REQUIRE(m >= 1 && n >= 1, "qr: empty matrix");
  const int k = std::min(m, n);
  T* Vall = ar.alloc<T>((size_t)m * k);
  const int nblk = (k + NB - 1) / NB;
  T* Tall = ar.alloc<T>((size_t)NB * NB * nblk);
  T* W1 = ar.alloc<T>((size_t)NB * std::max(n, k));
  T* W2 = ar.alloc<T>((size_t)NB * std::max(n, k));
  for (int b = 0; b < nblk; ++b) {
    const int j0 = b * NB, jb = std::min(NB, k - j0), mm = m - j0;
    T* Vb = Vall + j0 + (long long)j0 * m;
    T* Tb = Tall + (long long)b * NB * NB;
    // zero the rows above j0 of this block's V columns
    if (j0 > 0) {
      for (int c = 0; c < jb; ++c) QTT_CUDA(cudaMemsetAsync(Vall + (long long)(j0 + c) * m, 0, sizeof(T) * j0, s));
    }
    ProfToken pt = prof_begin(PROF_QR_PANEL, s);
    qr_panel_kernel<T><<<1, PT, 0, s>>>(mm, jb, A + j0 + (long long)j0 * lda, lda, Vb, m, Tb);
    QTT_CHECK_LAUNCH();
    if (pt.ev) prof_end(pt, s, 4.0 * mm * jb * jb, sizeof(T) * 3.0 * mm * jb);
    const int n2 = n - j0 - jb;
    if (n2 > 0) {
      T* C = A + j0 + (long long)(j0 + jb) * lda;
      gemm<T>(s, true, false, jb, n2, mm, T(1), Vb, m, 0, C, lda, 0, T(0), W1, jb, 0);
      gemm<T>(s, true, false, jb, n2, jb, T(1), Tb, NB, 0, W1, jb, 0, T(0), W2, jb, 0);
      gemm<T>(s, false, false, mm, n2, jb, T(-1), Vb, m, 0, W2, jb, 0, T(1), C, lda, 0);
    }
  }
  if (R) {
    upper_copy_kernel<T><<<grid_for((long long)k * n), 256, 0, s>>>(A, lda, R, ldr, k, n);
    QTT_CHECK_LAUNCH();
  }
  if (Q) {
    set_identity_kernel<T><<<grid_for((long long)m * k), 256, 0, s>>>(Q, m, k, ldq);
    QTT_CHECK_LAUNCH();
    for (int b = nblk - 1; b >= 0; --b) {
      const int j0 = b * NB, jb = std::min(NB, k - j0), mm = m - j0, nc = k - j0;
      T* Vb = Vall + j0 + (long long)j0 * m;
      T* Tb = Tall + (long long)b * NB * NB;
      T* Qs = Q + j0 + (long long)j0 * ldq;
      gemm<T>(s, true, false, jb, nc, mm, T(1), Vb, m, 0, Qs, ldq, 0, T(0), W1, jb, 0);
      gemm<T>(s, false, false, jb, nc, jb, T(1), Tb, NB, 0, W1, jb, 0, T(0), W2, jb, 0);
      gemm<T>(s, false, false, mm, nc, jb, T(-1), Vb, m, 0, W2, jb, 0, T(1), Qs, ldq, 0);
    }
  }
}

template <typename T>
void svd(cudaStream_t s, Arena& ar, int m, int n, T* A, int lda, T* U, int ldu, T* S, T* Vt, int ldvt) {
  QTT_REQUIRE(m >= 1 && n >= 1, "svd: empty matrix");
  if (m < n) {
    // SVD of A^T: A^T = U' S V'^T  =>  A = V' S U'^T
    T* At = ar.alloc<T>((size_t)n * m);
    int dims[2] = {m, n}, perm[2] = {1, 0};
    if (lda == m) {
      permute<T>(s, A, At, 2, dims, perm);
    } else {
      T* Ac = ar.alloc<T>((size_t)m * n);
      copy2d<T>(s, m, n, A, lda, Ac, m);
      permute<T>(s, Ac, At, 2, dims, perm);
    }
    const int k = m;
    T* Ut = ar.alloc<T>((size_t)n * k);
    T* Vtt = ar.alloc<T>((size_t)k * m);
    svd<T>(s, ar, n, m, At, n, Ut, n, S, Vtt, k);
    // U = V'  (m x k) = Vtt^T ; Vt = U'^T (k x n)
    int d1[2] = {k, m}, d2[2] = {n, k};
    T* tmp1 = ar.alloc<T>((size_t)m * k);
    permute<T>(s, Vtt, tmp1, 2, d1, perm);
    copy2d<T>(s, m, k, tmp1, m, U, ldu);
    T* tmp2 = ar.alloc<T>((size_t)k * n);
    permute<T>(s, Ut, tmp2, 2, d2, perm);
    copy2d<T>(s, k, n, tmp2, k, Vt, ldvt);
    return;
  }
  const int k = n;
  T* Q = ar.alloc<T>((size_t)m * k);
  T* R = ar.alloc<T>((size_t)k * n);
  qr<T>(s, ar, m, n, A, lda, Q, m, R, k);
  T* Vm = ar.alloc<T>((size_t)n * n);
  set_identity_kernel<T><<<grid_for((long long)n * n), 256, 0, s>>>(Vm, n, n, n);
  QTT_CHECK_LAUNCH();
  static int coop_dev = -1;
  if (coop_dev < 0) {
    int dev = 0, v = 0;
    coop_dev = (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && v) ? 1 : 0;
    cudaGetLastError();
  }
  // With cooperative launch the FP64 sweeps run on many SMs from the start
  // (a round costs one grid barrier plus one pair per warp); the FP32
  // pre-sweeps below pay off only when the FP64 sweeps would share one SM.
  if (sizeof(T) == 8 && n >= 24 && !coop_dev) {
    // Mixed-precision preconditioning (one CTA runs the Jacobi sweeps, and
    // one SM has 1/64 of its FP32 rate in FP64): the sweeps run first in
    // FP32 on an FP32 copy of R, their rotations V32 are made orthogonal to
    // FP64 accuracy by two Newton-Schulz steps V <- V (3 I - V^T V) / 2, and
    // R <- R V.  The FP64 sweeps below then start from nearly orthogonal
    // columns and converge (quadratically) in a sweep or two.
    float* R32 = ar.alloc<float>((size_t)k * n);
    float* V32 = ar.alloc<float>((size_t)n * n);
    convert<T, float>(s, R, R32, (size_t)k * n);
    set_identity_kernel<float><<<grid_for((long long)n * n), 256, 0, s>>>(V32, n, n, n);
    QTT_CHECK_LAUNCH();
    ProfToken pf = prof_begin(PROF_JACOBI_F32, s);
    const size_t wbytes = sizeof(float) * (size_t)k * n, vbytes = sizeof(float) * (size_t)n * n;
    if (wbytes <= kJacobiSmem) {
      static bool attr = false;
      if (!attr) {
        QTT_CUDA(cudaFuncSetAttribute(jacobi_smem_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kJacobiSmem));
        attr = true;
      }
      const int vin = (wbytes + vbytes <= kJacobiSmem) ? 1 : 0;
      jacobi_smem_kernel<float, float><<<1, 1024, wbytes + (vin ? vbytes : 0), s>>>(k, n, R32, k, V32, n, 40, vin);
    } else {
      jacobi_kernel<float, float><<<1, 1024, 0, s>>>(k, n, R32, k, V32, n, 40, nullptr);
    }
    QTT_CHECK_LAUNCH();
    if (pf.ev) prof_end(pf, s, 0.5 * n * (n - 1) * (6.0 * k + 12.0 * k + 12.0 * n), 4.0 * 2.0 * (k + n) * n);
    T* V0 = ar.alloc<T>((size_t)n * n);
    T* X = ar.alloc<T>((size_t)n * n);
    T* V1 = ar.alloc<T>((size_t)n * n);
    convert<float, T>(s, V32, V0, (size_t)n * n);
    for (int it = 0; it < 2; ++it) {
      gemm<T>(s, true, false, n, n, n, T(1), V0, n, 0, V0, n, 0, T(0), X, n, 0);        // X = V^T V
      QTT_CUDA(cudaMemcpyAsync(V1, V0, sizeof(T) * n * n, cudaMemcpyDeviceToDevice, s));
      gemm<T>(s, false, false, n, n, n, T(-0.5), V0, n, 0, X, n, 0, T(1.5), V1, n, 0);   // V1 = 1.5 V - 0.5 V X
      std::swap(V0, V1);
    }
    T* W = ar.alloc<T>((size_t)k * n);
    gemm<T>(s, false, false, k, n, n, T(1), R, k, 0, V0, n, 0, T(0), W, k, 0);           // W = R V
    QTT_CUDA(cudaMemcpyAsync(R, W, sizeof(T) * k * n, cudaMemcpyDeviceToDevice, s));
    QTT_CUDA(cudaMemcpyAsync(Vm, V0, sizeof(T) * n * n, cudaMemcpyDeviceToDevice, s));
    // the FP64 sweeps accumulate their rotations in V2; Vm <- Vm V2 afterwards
    T* V2 = ar.alloc<T>((size_t)n * n);
    set_identity_kernel<T><<<grid_for((long long)n * n), 256, 0, s>>>(V2, n, n, n);
    QTT_CHECK_LAUNCH();
    ProfToken pj = prof_begin(PROF_JACOBI, s);
    jacobi_sweeps<T, double>(s, ar, k, n, R, k, V2, n, 40);
    if (pj.ev) prof_end(pj, s, 0.5 * n * (n - 1) * (6.0 * k + 12.0 * k + 12.0 * n), sizeof(T) * 2.0 * (k + n) * n);
    gemm<T>(s, false, false, n, n, n, T(1), V0, n, 0, V2, n, 0, T(0), Vm, n, 0);
  } else {
    ProfToken pj = prof_begin(sizeof(T) == 8 ? PROF_JACOBI : PROF_JACOBI_F32, s);
    jacobi_sweeps<T, double>(s, ar, k, n, R, k, Vm, n, 40);
    // nominal work of one sweep over all pairs (the sweep count is data dependent)
    if (pj.ev) prof_end(pj, s, 0.5 * n * (n - 1) * (6.0 * k + 12.0 * k + 12.0 * n), sizeof(T) * 2.0 * (k + n) * n);
  }
  int* order = ar.alloc<int>(n);
  svd_finish_kernel<T><<<1, 1024, sizeof(double) * n, s>>>(k, n, R, k, S, order);
  QTT_CHECK_LAUNCH();
  // U_R columns reordered, U = Q U_R
  T* UR = ar.alloc<T>((size_t)k * k);
  gather_cols_kernel<T><<<grid_for((long long)k * k), 256, 0, s>>>(R, k, UR, k, k, k, order, false);
  QTT_CHECK_LAUNCH();
  gemm<T>(s, false, false, m, k, k, T(1), Q, m, 0, UR, k, 0, T(0), U, ldu, 0);
  // Vt = V^T with columns reordered
  gather_cols_kernel<T><<<grid_for((long long)n * k), 256, 0, s>>>(Vm, n, Vt, ldvt, n, k, order, true);
  QTT_CHECK_LAUNCH();
}

template <typename T>
void lu_solve(cudaStream_t s, Arena& ar, int n, T* A, int lda, T* B, int ldb, int nrhs, int* info) {
  QTT_REQUIRE(n >= 1, "lu_solve: empty system");
  if (info) QTT_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int jb = std::min(NB, n - j0);
    ProfToken pl = prof_begin(PROF_LU_PANEL, s);
    lu_panel_kernel<T><<<1, PT, 0, s>>>(n, j0, jb, A, lda, B, ldb, nrhs, info);
    QTT_CHECK_LAUNCH();
    if (pl.ev) prof_end(pl, s, 1.0 * (n - j0) * jb * jb, sizeof(T) * 2.0 * (n - j0) * jb);
    const int n2 = n - j0 - jb;
    if (n2 > 0) {
      T* L11 = A + j0 + (long long)j0 * lda;
      T* A12 = A + j0 + (long long)(j0 + jb) * lda;
      trsm_lower_unit_kernel<T><<<(n2 + 127) / 128, 128, 0, s>>>(jb, L11, lda, A12, lda, n2);
      QTT_CHECK_LAUNCH();
      T* L21 = A + (j0 + jb) + (long long)j0 * lda;
      T* A22 = A + (j0 + jb) + (long long)(j0 + jb) * lda;
      gemm<T>(s, false, false, n2, n2, jb, T(-1), L21, lda, 0, A12, lda, 0, T(1), A22, lda, 0);
    }
  }
  // forward: L y = B (unit lower), blocked
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int jb = std::min(NB, n - j0);
    trsv_block_kernel<T><<<(nrhs + 63) / 64, 64, 0, s>>>(jb, A + j0 + (long long)j0 * lda, lda, B + j0, ldb, nrhs,
                                                         false);
    QTT_CHECK_LAUNCH();
    const int n2 = n - j0 - jb;
    if (n2 > 0)
      gemm<T>(s, false, false, n2, nrhs, jb, T(-1), A + (j0 + jb) + (long long)j0 * lda, lda, 0, B + j0, ldb, 0,
              T(1), B + j0 + jb, ldb, 0);
  }
  // backward: U x = y
  const int nblk = (n + NB - 1) / NB;
  for (int b = nblk - 1; b >= 0; --b) {
    const int j0 = b * NB, jb = std::min(NB, n - j0);
    trsv_block_kernel<T><<<(nrhs + 63) / 64, 64, 0, s>>>(jb, A + j0 + (long long)j0 * lda, lda, B + j0, ldb, nrhs,
                                                         true);
    QTT_CHECK_LAUNCH();
    if (j0 > 0)
      gemm<T>(s, false, false, j0, nrhs, jb, T(-1), A + (long long)j0 * lda, lda, 0, B + j0, ldb, 0, T(1), B, ldb,
              0);
  }
}

template void qr<double>(cudaStream_t, Arena&, int, int, double*, int, double*, int, double*, int);
template void qr<float>(cudaStream_t, Arena&, int, int, float*, int, float*, int, float*, int);
template void svd<double>(cudaStream_t, Arena&, int, int, double*, int, double*, int, double*, double*, int);
template void svd<float>(cudaStream_t, Arena&, int, int, float*, int, float*, int, float*, float*, int);
template void lu_solve<double>(cudaStream_t, Arena&, int, double*, int, double*, int, int, int*);
template void lu_solve<float>(cudaStream_t, Arena&, int, float*, int, float*, int, int, int*);

}  // namespace qtt
