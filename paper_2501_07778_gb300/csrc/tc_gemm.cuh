// Tensor-core (tcgen05) FP32-accurate GEMM: declarations shared by the
// contraction code that uses it (tc_gemm.cu holds the kernel).
#pragma once

#include "common.cuh"

namespace qtt {

// offset of logical index idx = sum_t digit_t(idx) * s[t], digits of sizes n[t]
// (first fastest), up to four digits
struct TcIdxMap {
  int cnt;
  int n[4];
  long long s[4];
};

// where D[m, n] goes: out[om(m) + on(n)]; with lo != NULL the value is
// stored as a TF32 pair (out = hi, lo = v - hi) for a following tf32x3 GEMM;
// with atomic != 0 it is added to out (split K; FP32 output only)
struct TcEpilogue {
  TcIdxMap om, on;
  float* out;
  float* lo;
  int atomic;
};

// A GEMM whose operand buffers stay fixed over many launches (the Krylov
// iterations of one local solve): tensor maps encoded once.
struct TcGemmPlan {
  alignas(64) unsigned char maps[4][128];   // CUtensorMap of A_hi, A_lo, B_hi, B_lo
  int M, N, K, splits, kb_per;
  TcEpilogue epi;
};

// plan D = A B^T (TF32 pairs, K-major, ld multiples of 4) with the K loop
// split over up to max_splits CTAs per output tile (atomic epilogue when > 1)
void tc_plan(TcGemmPlan& p, int M, int N, int K, const float* Ahi, const float* Alo, int lda, const float* Bhi,
             const float* Blo, int ldb, const TcEpilogue& epi, int max_splits);
void tc_run(cudaStream_t s, const TcGemmPlan& p, int* err);

// the device is sm_103 and the TMA descriptor encoder is reachable
bool tc_available();

// hi = TF32(x), lo = x - hi, elementwise
void tf32_split(cudaStream_t s, const float* x, float* hi, float* lo, long long n);

// TF32 pairs of a rows x K K-major operand (leading dimension ld) gathered
// from src: element (row, k) = src[rmap(row) + kmap(k)]
void tc_pack(cudaStream_t s, const float* src, int rows, int K, int ld, const TcIdxMap& rmap, const TcIdxMap& kmap,
             float* hi, float* lo);

// D[m, n] = sum_k A[m, k] B[n, k] from TF32 pairs of A (M x K, K-major,
// leading dimension lda) and B (N x K, K-major, ldb); lda and ldb multiples
// of 4 elements, operands 16-byte aligned.  *err (device) receives
// QTT_ETIMEOUT if a bounded wait gave up.
void tf32x3_gemm(cudaStream_t s, int M, int N, int K, const float* Ahi, const float* Alo, int lda, const float* Bhi,
                 const float* Blo, int ldb, const TcEpilogue& epi, int* err);

}  // namespace qtt
