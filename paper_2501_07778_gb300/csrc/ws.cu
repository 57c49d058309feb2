// Learned warm start: a 3-layer MLP (tanh) from load/material features to
// fixed-rank QTT cores, its backward pass, the gauge-invariant TT loss and
// an Adam step -- all FP32 kernels of this library (column-major matrices,
// per-sample vectors contiguous).
//
//   a1 = W1 phi + b1, h1 = tanh(a1); a2 = W2 h1 + b2, h2 = tanh(a2);
//   out = W3 h2 + b3;  X_hat = TT(out) with rank-r cores cut in order.
//   loss_b = ||X_hat - X_b||^2 / ||X_b||^2 with X_b = sum_t c[b,t] basis_t,
//   evaluated through TT inner products (left/right transfer matrices), so
//   it does not depend on the gauge of the predicted cores.
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "common.cuh"

namespace qtt {
namespace {

inline int grid_for(long long n) { return grid_for_n(n, 32); }

__global__ void bias_tanh_kernel(float* a, const float* b, int H, int B) {
  long long total = (long long)H * B;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    a[t] = tanhf(a[t] + b[t % H]);
}

__global__ void bias_add_kernel(float* a, const float* b, int H, int B) {
  long long total = (long long)H * B;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    a[t] += b[t % H];
}

// g = g * (1 - h^2)
__global__ void tanh_back_kernel(float* g, const float* h, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    g[t] *= 1.0f - h[t] * h[t];
}

// row sums of a (H x B) column-major matrix -> out (H)
__global__ void rowsum_kernel(const float* a, int H, int B, float* out) {
  int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= H) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += a[h + (long long)H * b];
  out[h] = s;
}

__global__ void adam_kernel(int n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

template <typename S, typename D>
__global__ void scale_convert_kernel(const S* src, D* dst, long long n, double a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (D)(a * (double)src[i]);
}

}  // namespace

// TT inner-product environments on the device (FP32): L[k] (rx_k x ry_k)
struct Envs {
  std::vector<float*> L, R;
};

static void tt_envs(cudaStream_t s, Arena& ar, int d, const int* modes, const float* const* X, const int* rx,
                    const float* const* Y, const int* ry, Envs& e) {
  e.L.assign(d + 1, nullptr);
  e.R.assign(d + 1, nullptr);
  e.L[0] = ar.alloc<float>(1);
  fill<float>(s, e.L[0], 1, 1.f);
  for (int k = 0; k < d; ++k) {
    int n = modes[k];
    int dL[2] = {rx[k], ry[k]}, dX[3] = {rx[k], n, rx[k + 1]}, dY[3] = {ry[k], n, ry[k + 1]};
    float* t = ar.alloc<float>((size_t)ry[k] * n * rx[k + 1]);
    einsum<float>(s, ar, "ab,aic->bic", e.L[k], dL, X[k], dX, t);
    int dt[3] = {ry[k], n, rx[k + 1]};
    e.L[k + 1] = ar.alloc<float>((size_t)rx[k + 1] * ry[k + 1]);
    einsum<float>(s, ar, "bic,bid->cd", t, dt, Y[k], dY, e.L[k + 1]);
  }
  e.R[d] = ar.alloc<float>(1);
  fill<float>(s, e.R[d], 1, 1.f);
  for (int k = d - 1; k >= 0; --k) {
    int n = modes[k];
    int dR[2] = {rx[k + 1], ry[k + 1]}, dX[3] = {rx[k], n, rx[k + 1]}, dY[3] = {ry[k], n, ry[k + 1]};
    float* t = ar.alloc<float>((size_t)ry[k] * n * rx[k + 1]);
    einsum<float>(s, ar, "bid,cd->bic", Y[k], dY, e.R[k + 1], dR, t);
    int dt[3] = {ry[k], n, rx[k + 1]};
    e.R[k] = ar.alloc<float>((size_t)rx[k] * ry[k]);
    einsum<float>(s, ar, "aic,bic->ab", X[k], dX, t, dt, e.R[k]);
  }
}

// G += alpha * L[k] Y_k R[k+1]  (G shaped like X_k)
static void env_grad(cudaStream_t s, Arena& ar, int k, int n, const int* rx, const int* ry, const Envs& e,
                     const float* Yk, float alpha, float* G) {
  int dL[2] = {rx[k], ry[k]}, dY[3] = {ry[k], n, ry[k + 1]};
  float* t = ar.alloc<float>((size_t)rx[k] * n * ry[k + 1]);
  einsum<float>(s, ar, "ab,bid->aid", e.L[k], dL, Yk, dY, t);
  int dt[3] = {rx[k], n, ry[k + 1]}, dR[2] = {rx[k + 1], ry[k + 1]};
  einsum<float>(s, ar, "aid,cd->aic", t, dt, e.R[k + 1], dR, G, alpha, 1.f);
}

static float read_scalar(cudaStream_t s, const float* p) {
  float h = 0.f;
  QTT_CUDA(cudaMemcpyAsync(&h, p, sizeof(float), cudaMemcpyDeviceToHost, s));
  QTT_CUDA(cudaStreamSynchronize(s));
  return h;
}

}  // namespace qtt

using namespace qtt;

#define WS_BEGIN try {
#define WS_END                                   \
  }                                              \
  catch (const QttError& e) {                    \
    set_last_error(e.what());                    \
    return e.code;                               \
  }                                              \
  catch (const std::exception& e) {              \
    set_last_error(e.what());                    \
    return QTT_EINVAL;                           \
  }

extern "C" {

int qtt_ws_forward(int B, int nin, int H, int P, const float* W1, const float* b1, const float* W2, const float* b2,
                   const float* W3, const float* b3, const float* phi, float* h1, float* h2, float* out,
                   void* stream) {
  WS_BEGIN
  QTT_REQUIRE(B > 0 && nin > 0 && H > 0 && P > 0, "qtt_ws_forward: sizes must be positive");
  QTT_REQUIRE(W1 && b1 && W2 && b2 && W3 && b3 && phi && h1 && h2 && out, "qtt_ws_forward: null pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  gemm<float>(s, false, false, H, B, nin, 1.f, W1, H, 0, phi, nin, 0, 0.f, h1, H, 0);
  bias_tanh_kernel<<<grid_for((long long)H * B), 256, 0, s>>>(h1, b1, H, B);
  QTT_CHECK_LAUNCH();
  gemm<float>(s, false, false, H, B, H, 1.f, W2, H, 0, h1, H, 0, 0.f, h2, H, 0);
  bias_tanh_kernel<<<grid_for((long long)H * B), 256, 0, s>>>(h2, b2, H, B);
  QTT_CHECK_LAUNCH();
  gemm<float>(s, false, false, P, B, H, 1.f, W3, P, 0, h2, H, 0, 0.f, out, P, 0);
  bias_add_kernel<<<grid_for((long long)P * B), 256, 0, s>>>(out, b3, P, B);
  QTT_CHECK_LAUNCH();
  return QTT_OK;
  WS_END
}

int qtt_ws_backward(int B, int nin, int H, int P, const float* W2, const float* W3, const float* phi,
                    const float* h1, const float* h2, const float* gout, float* gW1, float* gb1, float* gW2,
                    float* gb2, float* gW3, float* gb3, float* work, void* stream) {
  WS_BEGIN
  QTT_REQUIRE(B > 0 && nin > 0 && H > 0 && P > 0, "qtt_ws_backward: sizes must be positive");
  QTT_REQUIRE(W2 && W3 && phi && h1 && h2 && gout && gW1 && gb1 && gW2 && gb2 && gW3 && gb3 && work,
              "qtt_ws_backward: null pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float* g2 = work;                     // H x B
  float* g1 = work + (size_t)H * B;     // H x B
  // gW3 = gout h2^T, gb3 = rowsum(gout)
  gemm<float>(s, false, true, P, H, B, 1.f, gout, P, 0, h2, H, 0, 0.f, gW3, P, 0);
  rowsum_kernel<<<(P + 255) / 256, 256, 0, s>>>(gout, P, B, gb3);
  QTT_CHECK_LAUNCH();
  // g2 = (W3^T gout) * (1 - h2^2)
  gemm<float>(s, true, false, H, B, P, 1.f, W3, P, 0, gout, P, 0, 0.f, g2, H, 0);
  tanh_back_kernel<<<grid_for((long long)H * B), 256, 0, s>>>(g2, h2, (long long)H * B);
  QTT_CHECK_LAUNCH();
  gemm<float>(s, false, true, H, H, B, 1.f, g2, H, 0, h1, H, 0, 0.f, gW2, H, 0);
  rowsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(g2, H, B, gb2);
  QTT_CHECK_LAUNCH();
  // g1 = (W2^T g2) * (1 - h1^2)
  gemm<float>(s, true, false, H, B, H, 1.f, W2, H, 0, g2, H, 0, 0.f, g1, H, 0);
  tanh_back_kernel<<<grid_for((long long)H * B), 256, 0, s>>>(g1, h1, (long long)H * B);
  QTT_CHECK_LAUNCH();
  gemm<float>(s, false, true, H, nin, B, 1.f, g1, H, 0, phi, nin, 0, 0.f, gW1, H, 0);
  rowsum_kernel<<<(H + 255) / 256, 256, 0, s>>>(g1, H, B, gb1);
  QTT_CHECK_LAUNCH();
  return QTT_OK;
  WS_END
}

int qtt_ws_basis_gram(int d, int nbasis, const qtt_tensor* const* basis, double* gram, void* stream) {
  WS_BEGIN
  QTT_REQUIRE(d >= 1 && nbasis >= 1 && basis && gram, "qtt_ws_basis_gram: bad argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int t = 0; t < nbasis; ++t) QTT_REQUIRE(basis[t] && basis[t]->prec == QTT_F32 && basis[t]->d == d, "qtt_ws_basis_gram: basis must be FP32 of length d");
  for (int t = 0; t < nbasis; ++t)
    for (int u = t; u < nbasis; ++u) {
      Arena a2(s);
      Envs e;
      tt_envs(s, a2, d, basis[t]->n, (const float* const*)basis[t]->core, basis[t]->r, (const float* const*)basis[u]->core,
              basis[u]->r, e);
      gram[t * nbasis + u] = gram[u * nbasis + t] = (double)read_scalar(s, e.L[d]);
    }
  return QTT_OK;
  WS_END
}

int qtt_ws_tt_loss(int B, int d, const int* modes, int r, const float* out, int nbasis,
                   const qtt_tensor* const* basis, const double* coef, const double* gram_in, float* loss,
                   float* gout, void* stream) {
  WS_BEGIN
  QTT_REQUIRE(B > 0 && d >= 1 && d <= QTT_MAX_CORES && r >= 1 && nbasis >= 1, "qtt_ws_tt_loss: bad sizes");
  QTT_REQUIRE(modes && out && basis && coef && loss && gout, "qtt_ws_tt_loss: null pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int t = 0; t < nbasis; ++t) {
    QTT_REQUIRE(basis[t] && basis[t]->prec == QTT_F32 && basis[t]->d == d, "qtt_ws_tt_loss: basis must be FP32 of length d");
    for (int k = 0; k < d; ++k) QTT_REQUIRE(basis[t]->n[k] == modes[k], "qtt_ws_tt_loss: basis modes differ");
  }
  std::vector<int> rx(d + 1, r);
  rx[0] = rx[d] = 1;
  std::vector<long long> off(d + 1, 0);
  for (int k = 0; k < d; ++k) off[k + 1] = off[k] + (long long)rx[k] * modes[k] * rx[k + 1];
  const long long P = off[d];
  Arena ar(s);
  // Gram of the basis: G[t, u] = <basis_t, basis_u> (given, or computed here)
  std::vector<double> gram((size_t)nbasis * nbasis, 0.0);
  if (gram_in) {
    for (size_t i = 0; i < gram.size(); ++i) gram[i] = gram_in[i];
  } else {
    int rc = qtt_ws_basis_gram(d, nbasis, basis, gram.data(), stream);
    if (rc != QTT_OK) return rc;
  }
  std::vector<float> hloss(B);
  for (int b = 0; b < B; ++b) {
    Arena sb(s);
    const float* o = out + P * b;
    float* g = gout + P * b;
    std::vector<const float*> Xc(d);
    for (int k = 0; k < d; ++k) Xc[k] = o + off[k];
    double xx = 0.0;
    for (int t = 0; t < nbasis; ++t)
      for (int u = 0; u < nbasis; ++u) xx += coef[b * nbasis + t] * coef[b * nbasis + u] * gram[t * nbasis + u];
    QTT_REQUIRE(xx > 0, "qtt_ws_tt_loss: zero target");
    Envs ehh;
    tt_envs(s, sb, d, modes, Xc.data(), rx.data(), Xc.data(), rx.data(), ehh);
    const double hh = read_scalar(s, ehh.L[d]);
    QTT_CUDA(cudaMemsetAsync(g, 0, sizeof(float) * P, s));
    for (int k = 0; k < d; ++k)
      env_grad(s, sb, k, modes[k], rx.data(), rx.data(), ehh, Xc[k], (float)(2.0 / xx), g + off[k]);
    double hx = 0.0;
    for (int t = 0; t < nbasis; ++t) {
      const double c = coef[b * nbasis + t];
      if (c == 0.0) continue;
      Envs ehx;
      tt_envs(s, sb, d, modes, Xc.data(), rx.data(), (const float* const*)basis[t]->core, basis[t]->r, ehx);
      hx += c * (double)read_scalar(s, ehx.L[d]);
      for (int k = 0; k < d; ++k)
        env_grad(s, sb, k, modes[k], rx.data(), basis[t]->r, ehx, (const float*)basis[t]->core[k],
                 (float)(-2.0 * c / xx), g + off[k]);
    }
    hloss[b] = (float)((hh - 2.0 * hx + xx) / xx);
    // the mean over the batch is the training objective
    axpby<float>(s, (size_t)P, 1.0f / B, g, 0.f, g);
  }
  QTT_CUDA(cudaMemcpyAsync(loss, hloss.data(), sizeof(float) * B, cudaMemcpyHostToDevice, s));
  QTT_CUDA(cudaStreamSynchronize(s));
  return QTT_OK;
  WS_END
}

int qtt_ws_adam(int n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2, float eps, int t,
                void* stream) {
  WS_BEGIN
  QTT_REQUIRE(n > 0 && w && g && m && v && t >= 1, "qtt_ws_adam: bad argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<grid_for(n), 256, 0, s>>>(n, w, g, m, v, lr, b1, b2, eps, c1, c2);
  QTT_CHECK_LAUNCH();
  return QTT_OK;
  WS_END
}

int qtt_ws_to_tensor(const float* out_row, int d, const int* modes, int r, double scale, qtt_tensor** x,
                     void* stream) {
  WS_BEGIN
  QTT_REQUIRE(out_row && modes && x && d >= 1 && d <= QTT_MAX_CORES && r >= 1, "qtt_ws_to_tensor: bad argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  StreamScope scope_(s);
  std::vector<int> rr(d + 1, r);
  rr[0] = rr[d] = 1;
  qtt_tensor* t = tensor_alloc(d, modes, nullptr, rr.data(), QTT_F64, 0);
  long long off = 0;
  for (int k = 0; k < d; ++k) {
    long long e = (long long)rr[k] * modes[k] * rr[k + 1];
    scale_convert_kernel<float, double><<<grid_for(e), 256, 0, s>>>(out_row + off, (double*)t->core[k], e,
                                                                    k == 0 ? scale : 1.0);
    QTT_CHECK_LAUNCH();
    off += e;
  }
  *x = t;
  return QTT_OK;
  WS_END
}

}  // extern "C"
