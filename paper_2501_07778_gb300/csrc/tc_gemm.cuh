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
// stored as a TF32 pair (out = hi, lo = v - hi) for a following tf32x3 GEMM
struct TcEpilogue {
  TcIdxMap om, on;
  float* out;
  float* lo;
};

// the device is sm_103 and the TMA descriptor encoder is reachable
bool tc_available();

// hi = TF32(x), lo = x - hi, elementwise
void tf32_split(cudaStream_t s, const float* x, float* hi, float* lo, long long n);

// D[m, n] = sum_k A[m, k] B[n, k] from TF32 pairs of A (M x K, K-major,
// leading dimension lda) and B (N x K, K-major, ldb); lda and ldb multiples
// of 4 elements, operands 16-byte aligned.  *err (device) receives
// QTT_ETIMEOUT if a bounded wait gave up.
void tf32x3_gemm(cudaStream_t s, int M, int N, int K, const float* Ahi, const float* Alo, int lda, const float* Bhi,
                 const float* Blo, int ldb, const TcEpilogue& epi, int* err);

}  // namespace qtt
