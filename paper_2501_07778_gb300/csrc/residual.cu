// Rounded FP64 residual r = f - K u for the outer iterative refinement.
//
// Forming K u exactly gives cores of rank R r + p (about 3400 for a
// single-patch plate at L = 12), and the QR sweep of the deterministic
// rounding then costs O(D (R r)^3) FP64 flops, more than a whole solve.
// Instead the residual is rounded by randomize-then-orthogonalize (Al Daas,
// Ballard, Cazeaux, Hallman, Miedlar, Pasha, Reid and Saibaba, "Randomized
// algorithms for rounding in the Tensor-Train format", SIAM J. Sci. Comput.
// 2023), applied to the structured sum f - K u so that the product cores are
// never formed:
//   1. right-to-left sketches W_b = (cores b..D-1 of r) x (cores of a
//      Gaussian TT G of rank ell), computed separately for f and for K u
//      (the K u sketch contracts u, then K, then G, one core at a time);
//   2. left to right: project the next core of r onto the orthonormal
//      left factor built so far (M_k), multiply by the sketch W_{k+1},
//      QR the (q_k n) x ell result; its Q is the output core k.
// The result is the orthogonal projection of r onto the span of its left
// factors, so ||r - r~||^2 = ||r||^2 - ||r~||^2, and ||r~|| is the norm of
// its last core (the others are left-orthonormal).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "tt_ops.cuh"

namespace qtt {
namespace {

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) on a counter, then Box-Muller to N(0, 1).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void gaussian_kernel(double* out, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long a = mix64(seed ^ mix64(2ULL * (unsigned long long)i));
    const unsigned long long b = mix64(seed ^ mix64(2ULL * (unsigned long long)i + 1ULL));
    const double u1 = ((double)(a >> 11) + 1.0) * (1.0 / 9007199254740993.0);   // (0, 1]
    const double u2 = (double)(b >> 11) * (1.0 / 9007199254740992.0);           // [0, 1)
    out[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

__global__ void set_scalar_kernel(double* p, double v) { *p = v; }

inline int blocks_for(long long n) { return grid_for_n(n, 8); }

}  // namespace

qtt_tensor* round_residual_rand(cudaStream_t s, const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f,
                                int ell, unsigned long long seed, double* kept_norm) {
  QTT_REQUIRE(K && u && f, "round_residual_rand: null operand");
  QTT_REQUIRE(K->prec == QTT_F64 && u->prec == QTT_F64 && f->prec == QTT_F64,
              "round_residual_rand: operands must be FP64");
  QTT_REQUIRE(K->is_matrix && !u->is_matrix && !f->is_matrix && K->d == u->d && K->d == f->d,
              "round_residual_rand: K must be an MPO and u, f MPS of equal length");
  const int D = K->d;
  for (int k = 0; k < D; ++k)
    QTT_REQUIRE(K->n[k] == f->n[k] && K->m[k] == u->n[k], "round_residual_rand: mode sizes differ");
  QTT_REQUIRE(ell >= 1, "round_residual_rand: sketch rank must be positive");
  Arena ar(s);
  // sketch ranks: bounded by ell, by the rank of r and by the mode products
  std::vector<int> lr(D + 1, 1);
  {
    std::vector<double> left(D + 1, 1.0), right(D + 1, 1.0);
    for (int k = 0; k < D; ++k) left[k + 1] = std::min(1e18, left[k] * K->n[k]);
    for (int k = D - 1; k >= 0; --k) right[k] = std::min(1e18, right[k + 1] * K->n[k]);
    for (int b = 1; b < D; ++b) {
      const double rr = (double)K->r[b] * u->r[b] + f->r[b];
      lr[b] = (int)std::max(1.0, std::min(std::min((double)ell, rr), std::min(left[b], right[b])));
    }
  }
  // Gaussian TT cores G_b: (lr[b], n_b, lr[b+1])
  std::vector<double*> G(D, nullptr);
  for (int b = 1; b < D; ++b) {
    const long long e = (long long)lr[b] * K->n[b] * lr[b + 1];
    G[b] = ar.alloc<double>(e);
    gaussian_kernel<<<blocks_for(e), 256, 0, s>>>(G[b], e, seed * 0x2545F4914F6CDD1DULL + (unsigned long long)b);
    QTT_CHECK_LAUNCH();
  }
  // right-to-left sketches; Wk[b]: (R_b, r_b, lr[b]) and Wf[b]: (p_b, lr[b])
  std::vector<double*> Wk(D + 1, nullptr), Wf(D + 1, nullptr);
  Wk[D] = ar.alloc<double>(1);
  Wf[D] = ar.alloc<double>(1);
  fill<double>(s, Wk[D], 1, 1.0);
  fill<double>(s, Wf[D], 1, 1.0);
  for (int b = D - 1; b >= 1; --b) {
    const int n = K->n[b], Ra = K->r[b], Rb = K->r[b + 1], ra = u->r[b], rb = u->r[b + 1];
    const int pa = f->r[b], pb = f->r[b + 1], la = lr[b], lb = lr[b + 1];
    // K u part: cjd,bdm->cjbm ; cjbm,aijb->cmai ; cmai,lim->acl
    double* T1 = ar.alloc<double>((size_t)ra * n * Rb * lb);
    int du[3] = {ra, n, rb}, dW[3] = {Rb, rb, lb};
    einsum<double>(s, ar, "cjd,bdm->cjbm", (const double*)u->core[b], du, Wk[b + 1], dW, T1);
    double* T2 = ar.alloc<double>((size_t)ra * lb * Ra * n);
    int d1[4] = {ra, n, Rb, lb}, dK[4] = {Ra, n, n, Rb};
    einsum<double>(s, ar, "cjbm,aijb->cmai", T1, d1, (const double*)K->core[b], dK, T2);
    Wk[b] = ar.alloc<double>((size_t)Ra * ra * la);
    int d2[4] = {ra, lb, Ra, n}, dG[3] = {la, n, lb};
    einsum<double>(s, ar, "cmai,lim->acl", T2, d2, G[b], dG, Wk[b]);
    // f part: eig,gm->eim ; eim,lim->el
    double* T3 = ar.alloc<double>((size_t)pa * n * lb);
    int df[3] = {pa, n, pb}, dWf[2] = {pb, lb};
    einsum<double>(s, ar, "eig,gm->eim", (const double*)f->core[b], df, Wf[b + 1], dWf, T3);
    Wf[b] = ar.alloc<double>((size_t)pa * la);
    int d3[3] = {pa, n, lb};
    einsum<double>(s, ar, "eim,lim->el", T3, d3, G[b], dG, Wf[b]);
  }
  // left to right
  std::vector<int> q(D + 1, 1);
  std::vector<int> nn(D);
  for (int k = 0; k < D; ++k) nn[k] = K->n[k];
  // output ranks are only known as we go: build cores in scratch, copy at the end
  std::vector<double*> out(D, nullptr);
  double* Mk = ar.alloc<double>(1);   // (q_k, R_k, r_k)
  double* Mf = ar.alloc<double>(1);   // (q_k, p_k)
  set_scalar_kernel<<<1, 1, 0, s>>>(Mk, -1.0);
  QTT_CHECK_LAUNCH();
  set_scalar_kernel<<<1, 1, 0, s>>>(Mf, 1.0);
  QTT_CHECK_LAUNCH();
  for (int k = 0; k < D; ++k) {
    const int n = K->n[k], Ra = K->r[k], Rb = K->r[k + 1], ra = u->r[k], rb = u->r[k + 1];
    const int pa = f->r[k], pb = f->r[k + 1], qa = q[k];
    // Y^f[q,i,g] = sum_e Mf[q,e] f_k[e,i,g]
    double* Yf = ar.alloc<double>((size_t)qa * n * pb);
    int dMf[2] = {qa, pa}, df[3] = {pa, n, pb};
    einsum<double>(s, ar, "qe,eig->qig", Mf, dMf, (const double*)f->core[k], df, Yf);
    // Y^Ku[q,i,b,d] = sum_{a,c,j} Mk[q,a,c] u_k[c,j,d] K_k[a,i,j,b]
    double* T = ar.alloc<double>((size_t)qa * Ra * n * rb);
    int dMk[3] = {qa, Ra, ra}, du[3] = {ra, n, rb};
    einsum<double>(s, ar, "qac,cjd->qajd", Mk, dMk, (const double*)u->core[k], du, T);
    double* Yk = ar.alloc<double>((size_t)qa * n * Rb * rb);
    int dT[4] = {qa, Ra, n, rb}, dK[4] = {Ra, n, n, Rb};
    einsum<double>(s, ar, "qajd,aijb->qibd", T, dT, (const double*)K->core[k], dK, Yk);
    if (k == D - 1) {
      // last core: Y^f + Y^Ku (trailing ranks are 1)
      out[k] = ar.alloc<double>((size_t)qa * n);
      QTT_CUDA(cudaMemcpyAsync(out[k], Yf, sizeof(double) * qa * n, cudaMemcpyDeviceToDevice, s));
      axpby<double>(s, (size_t)qa * n, 1.0, Yk, 1.0, out[k]);
      break;
    }
    const int lb = lr[k + 1];
    // Z[q,i,l] = Y^f W^f_{k+1} + Y^Ku W^Ku_{k+1}
    double* Z = ar.alloc<double>((size_t)qa * n * lb);
    int dYf[3] = {qa, n, pb}, dWf[2] = {pb, lb};
    einsum<double>(s, ar, "qig,gl->qil", Yf, dYf, Wf[k + 1], dWf, Z);
    int dYk[4] = {qa, n, Rb, rb}, dWk[3] = {Rb, rb, lb};
    einsum<double>(s, ar, "qibd,bdl->qil", Yk, dYk, Wk[k + 1], dWk, Z, 1.0, 1.0);
    const int rows = qa * n, qb = std::min(rows, lb);
    double* Q = ar.alloc<double>((size_t)rows * qb);
    double* R = ar.alloc<double>((size_t)qb * lb);
    qr<double>(s, ar, rows, lb, Z, rows, Q, rows, R, qb);
    out[k] = Q;
    q[k + 1] = qb;
    // project: Mf'[Q,g] = sum_{q,i} Q[q,i,Q] Y^f[q,i,g];  Mk'[Q,b,d] likewise
    double* Mf2 = ar.alloc<double>((size_t)qb * pb);
    int dQ[3] = {qa, n, qb};
    einsum<double>(s, ar, "qiQ,qig->Qg", Q, dQ, Yf, dYf, Mf2);
    double* Mk2 = ar.alloc<double>((size_t)qb * Rb * rb);
    einsum<double>(s, ar, "qiQ,qibd->Qbd", Q, dQ, Yk, dYk, Mk2);
    Mf = Mf2;
    Mk = Mk2;
  }
  std::vector<int> mm(D, 1);
  qtt_tensor* r = tensor_alloc(D, nn.data(), mm.data(), q.data(), QTT_F64, 0);
  try {
    for (int k = 0; k < D; ++k)
      QTT_CUDA(cudaMemcpyAsync(r->core[k], out[k], sizeof(double) * core_elems(r, k), cudaMemcpyDeviceToDevice, s));
    if (kept_norm) {
      double* dv = ar.alloc<double>(1);
      sumsq<double>(s, out[D - 1], core_elems(r, D - 1), dv);
      double v = 0;
      QTT_CUDA(cudaMemcpyAsync(&v, dv, sizeof(double), cudaMemcpyDeviceToHost, s));
      QTT_CUDA(cudaStreamSynchronize(s));
      *kept_norm = std::sqrt(v);
    } else {
      QTT_CUDA(cudaStreamSynchronize(s));
    }
  } catch (...) {
    tensor_free(r);
    throw;
  }
  return r;
}

}  // namespace qtt
