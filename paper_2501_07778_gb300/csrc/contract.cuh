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
  T As[2][CT_BK][TS + 1];     // two K blocks: one being read, the next being filled
  T Bs[2][CT_BK][TS + 1];
  long long rowA[TS], colB[TS], rowC[TS], colC[TS];
  long long kA[2][CT_BK], kB[2][CT_BK];
};

// One TS x TS output tile (TS = 64, or 32 for contractions too small to fill
// the SMs with 64 x 64 tiles) of work item `item` (tile_m, tile_n, batch,
// split flattened); all 256 threads of the block participate, each holding a
// (TS/16) x (TS/16) register tile.  The K loop is software-pipelined: the
// gathers of block k+1 are issued into registers (all of a thread's loads at
// once) before block k is multiplied out of shared memory, and a single
// barrier per block separates the two shared-memory buffers.  Operand and
// output offsets come from per-tile index tables, so the inner loops do no
// mixed-radix index arithmetic.
template <typename T, int TS = CT_BM>
__device__ void contract_tile(const ContractArgs& a, T alpha, const T* __restrict__ A, const T* __restrict__ B, T beta,
                              T* __restrict__ C, int item, ContractSmem<T, TS>& sm) {
  constexpr int R = TS / 16;                     // outputs per thread along each side
  static_assert((CT_BK * TS) % 256 == 0 && 4 * TS <= 256, "tile shape must match the 256-thread block");
  constexpr int LOADS = CT_BK * TS / 256;
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
  __syncthreads();   // the previous tile's readers of the tables and buffers are done
  if (tid < TS) {
    sm.rowA[tid] = (m0 + tid < a.M) ? idx_off(a.am, m0 + tid) : 0;
  } else if (tid < 2 * TS) {
    const int g = n0 + tid - TS;
    sm.colB[tid - TS] = (g < a.N) ? idx_off(a.bn, g) : 0;
  } else if (tid < 3 * TS) {
    const int g = m0 + tid - 2 * TS;
    sm.rowC[tid - 2 * TS] = (g < a.M) ? idx_off(a.cm, g) : 0;
  } else if (tid < 4 * TS) {
    const int g = n0 + tid - 3 * TS;
    sm.colC[tid - 3 * TS] = (g < a.N) ? idx_off(a.cn, g) : 0;
  }
  auto ktable = [&](int k0, int kbuf) {
    if (tid < CT_BK) sm.kA[kbuf][tid] = (k0 + tid < ke) ? idx_off(a.ak, k0 + tid) : 0;
    else if (tid < 2 * CT_BK) sm.kB[kbuf][tid - CT_BK] = (k0 + tid - CT_BK < ke) ? idx_off(a.bk, k0 + tid - CT_BK) : 0;
  };
  T va[LOADS], vb[LOADS];
  auto gather = [&](int k0, int kbuf) {
#pragma unroll
    for (int t = 0; t < LOADS; ++t) {
      const int L = tid + 256 * t;
      int i, k, j, kk;
      if (a.a_m_fast) { i = L % TS; k = L / TS; } else { k = L % CT_BK; i = L / CT_BK; }
      if (a.b_n_fast) { j = L % TS; kk = L / TS; } else { kk = L % CT_BK; j = L / CT_BK; }
      va[t] = (m0 + i < a.M && k0 + k < ke) ? A[sm.rowA[i] + sm.kA[kbuf][k]] : T(0);
      vb[t] = (n0 + j < a.N && k0 + kk < ke) ? B[sm.kB[kbuf][kk] + sm.colB[j]] : T(0);
    }
  };
  auto stage = [&](int buf) {
#pragma unroll
    for (int t = 0; t < LOADS; ++t) {
      const int L = tid + 256 * t;
      int i, k, j, kk;
      if (a.a_m_fast) { i = L % TS; k = L / TS; } else { k = L % CT_BK; i = L / CT_BK; }
      if (a.b_n_fast) { j = L % TS; kk = L / TS; } else { kk = L % CT_BK; j = L / CT_BK; }
      sm.As[buf][k][i] = va[t];
      sm.Bs[buf][kk][j] = vb[t];
    }
  };
  T acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = T(0);
  ktable(kb, 0);
  __syncthreads();
  if (kb < ke) gather(kb, 0);
  int buf = 0;
  for (int k0 = kb; k0 < ke; k0 += CT_BK) {
    // buffer `buf` was last read by the multiply two blocks back, and every
    // thread passed the previous barrier after finishing it
    stage(buf);
    const int kn = k0 + CT_BK;
    if (kn < ke) ktable(kn, buf ^ 1);
    __syncthreads();
    if (kn < ke) gather(kn, buf ^ 1);
#pragma unroll
    for (int k = 0; k < CT_BK; ++k) {
      T x[R], y[R];
#pragma unroll
      for (int i = 0; i < R; ++i) x[i] = sm.As[buf][k][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) y[j] = sm.Bs[buf][k][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
    }
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int gi = m0 + tx + 16 * i;
    if (gi >= a.M) continue;
    const long long ro = sm.rowC[tx + 16 * i];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int gj = n0 + ty + 16 * j;
      if (gj >= a.N) continue;
      T* c = C + ro + sm.colC[ty + 16 * j];
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
