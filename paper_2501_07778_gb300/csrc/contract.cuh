// Strided two-operand contraction: C[m, n] = alpha sum_k A[m, k] B[k, n] +
// beta C[m, n], where each logical index (m, n, k, batch) is a product of up
// to four tensor indices with arbitrary strides (column-major tensors, first
// index fastest).  A two-operand Einstein summation becomes one tiled GEMM
// with no transposed copies.  The tile routine is a device function so that
// persistent kernels can run several contractions between grid barriers.
#pragma once

#include <string>

#include "common.cuh"

namespace qtt {

constexpr int CT_BM = 64, CT_BN = 64, CT_BK = 16;

struct IdxMap {
  int cnt;
  int n[4];
  long long s[4];
};

struct ContractArgs {
  int M, N, K, batch;
  IdxMap am, ak, bk, bn, cm, cn, ab, bb, cb;
  bool a_m_fast, b_n_fast;   // which logical index runs along stride-1 memory
  int tile;                  // square output tile side (64, or 32 for small contractions)
  int tiles_m, tiles_n;      // output tiles per batch entry
  int splits, kchunk;        // K split (splits > 1: atomic accumulation into C)
};

__device__ __forceinline__ long long idx_off(const IdxMap& d, int idx) {
  long long o = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (t < d.cnt) {
      o += (long long)(idx % d.n[t]) * d.s[t];
      idx /= d.n[t];
    }
  }
  return o;
}

template <typename T, int TS = CT_BM>
struct ContractSmem {
  T As[CT_BK][TS + 1];
  T Bs[CT_BK][TS + 1];
  long long rowA[TS], colB[TS], kA[CT_BK], kB[CT_BK];
};

// One TS x TS output tile (TS = 64, or 32 for contractions too small to fill
// the SMs with 64 x 64 tiles) of work item `item` (tile_m, tile_n, batch,
// split flattened); all 256 threads of the block participate, each holding a
// (TS/16) x (TS/16) register tile.
template <typename T, int TS = CT_BM>
__device__ void contract_tile(const ContractArgs& a, T alpha, const T* __restrict__ A, const T* __restrict__ B, T beta,
                              T* __restrict__ C, int item, ContractSmem<T, TS>& sm) {
  constexpr int R = TS / 16;                     // outputs per thread along each side
  constexpr int LOADS = (CT_BK * TS + 255) / 256;
  const int tm = item % a.tiles_m;
  int rest = item / a.tiles_m;
  const int tn = rest % a.tiles_n;
  rest /= a.tiles_n;
  const int sp = rest % a.splits;
  const int bz = rest / a.splits;
  A += idx_off(a.ab, bz);
  B += idx_off(a.bb, bz);
  C += idx_off(a.cb, bz);
  const int kb = sp * a.kchunk, ke = min(a.K, kb + a.kchunk);
  const int m0 = tm * TS, n0 = tn * TS;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  __syncthreads();
  if (tid < TS) sm.rowA[tid] = (m0 + tid < a.M) ? idx_off(a.am, m0 + tid) : 0;
  else if (tid < 2 * TS) sm.colB[tid - TS] = (n0 + tid - TS < a.N) ? idx_off(a.bn, n0 + tid - TS) : 0;
  T acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = T(0);
  for (int k0 = kb; k0 < ke; k0 += CT_BK) {
    __syncthreads();
    if (tid < CT_BK) sm.kA[tid] = (k0 + tid < ke) ? idx_off(a.ak, k0 + tid) : 0;
    else if (tid < 2 * CT_BK) sm.kB[tid - CT_BK] = (k0 + tid - CT_BK < ke) ? idx_off(a.bk, k0 + tid - CT_BK) : 0;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < LOADS; ++t) {
      int L = tid + 256 * t;
      if (L >= CT_BK * TS) break;
      int i, k;
      if (a.a_m_fast) { i = L % TS; k = L / TS; } else { k = L % CT_BK; i = L / CT_BK; }
      T v = T(0);
      if (m0 + i < a.M && k0 + k < ke) v = A[sm.rowA[i] + sm.kA[k]];
      sm.As[k][i] = v;
      int j, kk;
      if (a.b_n_fast) { j = L % TS; kk = L / TS; } else { kk = L % CT_BK; j = L / CT_BK; }
      T w = T(0);
      if (n0 + j < a.N && k0 + kk < ke) w = B[sm.kB[kk] + sm.colB[j]];
      sm.Bs[kk][j] = w;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < CT_BK; ++k) {
      T x[R], y[R];
#pragma unroll
      for (int i = 0; i < R; ++i) x[i] = sm.As[k][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) y[j] = sm.Bs[k][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int gi = m0 + tx + 16 * i;
    if (gi >= a.M) continue;
    const long long ro = idx_off(a.cm, gi);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int gj = n0 + ty + 16 * j;
      if (gj >= a.N) continue;
      T* c = C + ro + idx_off(a.cn, gj);
      if (a.splits > 1) atomicAdd(c, alpha * acc[i][j]);
      else *c = (beta == T(0)) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*c);
    }
  }
}

// element t of the (M x N x batch) output -> its address offset
__device__ __forceinline__ long long contract_out_off(const ContractArgs& a, long long t) {
  int i = (int)(t % a.M);
  long long r = t / a.M;
  int j = (int)(r % a.N), b = (int)(r / a.N);
  return idx_off(a.cb, b) + idx_off(a.cm, i) + idx_off(a.cn, j);
}

// Host planner: parses "ab,bc->ac" style specs, classifies labels, builds
// the index maps and chooses the tile (32 x 32 when allow_small and 64 x 64
// tiles would leave work items below min_items) and the K split (min_items:
// target number of work items).  Returns false if a label group needs more
// than four indices.
bool plan_contract(const char* spec, const int* dA, const int* dB, int sizeof_T, long long min_items,
                   ContractArgs& ca, bool allow_small = false);

__host__ __device__ inline long long contract_items(const ContractArgs& a) {
  return (long long)a.tiles_m * a.tiles_n * a.splits * a.batch;
}

}  // namespace qtt
