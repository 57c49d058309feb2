// TT operations shared by the C ABI, the assembly and the solver.
#pragma once

#include <vector>

#include "common.cuh"

namespace qtt {

// Y_k = A_k (x) X_k core product (MPO x MPS when p = 1, MPO x MPO otherwise)
template <typename T>
void core_product(cudaStream_t s, int R0, int n, int mm, int R1, int r0, int p, int r1, const T* A, const T* X, T* Y);

template <typename T>
void to_full(cudaStream_t s, Arena& ar, const qtt_tensor* x, T* dst, size_t n_elems, int ordering);

// exact product (ranks multiply); new tensor
template <typename T>
qtt_tensor* product(cudaStream_t s, const qtt_tensor* A, const qtt_tensor* X);

// alpha X + beta Y (ranks add); new tensor
template <typename T>
qtt_tensor* tt_sum(cudaStream_t s, T alpha, const qtt_tensor* X, T beta, const qtt_tensor* Y);

// QR sweeps; cores [0, upto) left-orthonormal / cores (downto, d) right-orthonormal
template <typename T>
void left_orthogonalize(cudaStream_t s, Arena& ar, qtt_tensor* x, int upto);
template <typename T>
void right_orthogonalize(cudaStream_t s, Arena& ar, qtt_tensor* x, int downto);

template <typename T>
double norm(cudaStream_t s, Arena& ar, const qtt_tensor* x);

// smallest rank with discarded tail <= delta (capped at max_rank > 0)
int truncation_rank(const std::vector<double>& sv, double delta, int max_rank, bool* capped);

// in-place rounding; returns QTT_OK or QTT_ERANKCAP
template <typename T>
int round_tt(cudaStream_t s, Arena& ar, qtt_tensor* x, double tol, int max_rank);

// FP64 rank-ell approximation of f - K u by randomize-then-orthogonalize
// rounding of the structured sum (new tensor, left-orthonormal cores);
// *kept_norm = its norm.  The product cores of K u are never formed.
qtt_tensor* round_residual_rand(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f,
                                int ell, unsigned long long seed, double* kept_norm);

// canonical full vector (patch blocks of interleaved components
// 2 (i + n j) + c, 2 q 4^L entries) -> QTT (Z-block) order
template <typename T>
void from_canonical(cudaStream_t s, const T* in, T* out, int L, int q);

// TT-SVD of a full FP64 device vector in QTT order (first core's index
// fastest) with mode sizes n[0..d): new left-orthonormal tensor whose every
// unfolding drops a tail <= eps ||v|| / sqrt(d - 1), ranks capped at
// max_rank (> 0); meant for eps >= 1e-6 (Gram eigendecomposition of wide
// unfoldings)
qtt_tensor* tt_svd_full(cudaStream_t s, Arena& ar, const double* v, int d, const int* n, double eps, int max_rank);

// B = A diag(S)
template <typename T>
void scale_columns(cudaStream_t s, int rows, int cols, const T* A, int lda, const T* S, T* B, int ldb);

}  // namespace qtt
