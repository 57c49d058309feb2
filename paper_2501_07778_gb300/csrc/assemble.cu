// qtt_assemble_stiffness: Algorithm 1 on the device, in FP64.
//
// The paper assembles each patch matrix from element integrals moved into
// place by shift matrices V_c (Eq. Nodal:Stiffness:Matrix, summed over the
// sixteen corner pairs, Eq. Subdomain:Stiffness:Matrix).  On unit-square
// patches every element is the same square, so V_c1^T diag(k) V_c2 separates
// into 1D factors and the sixteen-term sum collapses to the textbook 1D Q1
// matrices:
//   S = (1/h)(2 I - P0 - PN - J - J^T)        stiffness  int phi_i' phi_k'
//   M = (h/6)(4 I - 2 P0 - 2 PN + J + J^T)     mass       int phi_i  phi_k
//   G = (1/2)(PN - P0 - J + J^T)               mixed      int phi_i' phi_k
// with J the superdiagonal shift and P0 / PN the corner projectors.  Their
// QTT cores are written in closed form (J by binary carry propagation, rank
// 2; the rest rank 1), and the 2D blocks follow by z-kron (Section 3.8):
//   K_xx = C11 S(x)M + C33 M(x)S,   K_yy = C22 M(x)S + C33 S(x)M,
//   K_xy = C12 G(x)G^T + C33 G^T(x)G,   K_yx = C12 G^T(x)G + C33 G(x)G^T.
// Concatenation (Section 3.6, read as: diagonal blocks K^(m) + gamma D_m,
// off-diagonal blocks Pi^(mp) K^(p) - gamma Pi^(mp), gamma on xx and yy
// only), component blocks (Section 3.7) and the Dirichlet masks (Section 3.8,
// K <- M K M + (I - M), f <- M f) are TT sums, products and Hadamard products
// followed by rounding.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "common.cuh"
#include "tt_ops.cuh"

namespace qtt {
namespace {

using Tptr = std::unique_ptr<qtt_tensor, void (*)(qtt_tensor*)>;
Tptr own(qtt_tensor* t) { return Tptr(t, tensor_free); }

inline int grid_for(long long n) { return grid_for_n(n, 32); }

// ---------------------------------------------------------------------------
// Closed-form 1D cores (LSB first).  Matrix cores are (r0, 2, 2, r1)
// column-major: element (a, i, i', b) at a + r0 (i + 2 (i' + 2 b)).
// ---------------------------------------------------------------------------
enum MatKind { M_I = 0, M_J = 1, M_JT = 2, M_P0 = 3, M_PN = 4, M_E10 = 5, M_E01 = 6 };

__global__ void mat1d_kernel(int kind, int k, int L, double* core, int r0, int r1) {
  int t = threadIdx.x;
  int total = r0 * 4 * r1;
  if (t >= total) return;
  int a = t % r0, i = (t / r0) % 2, ip = (t / (2 * r0)) % 2, b = t / (4 * r0);
  double v = 0.0;
  switch (kind) {
    case M_I: v = (i == ip); break;
    case M_P0: v = (i == 0 && ip == 0); break;
    case M_PN: v = (i == 1 && ip == 1); break;
    case M_E10: v = (i == 1 && ip == 0); break;     // row n-1, column 0
    case M_E01: v = (i == 0 && ip == 1); break;     // row 0, column n-1
    case M_J:
    case M_JT: {
      // column index = row index + 1 (J) or row index - 1 (J^T): carry c_in
      // from the less significant core, c_out to the next one
      int row = (kind == M_J) ? i : ip, col = (kind == M_J) ? ip : i;
      int cin = (k == 0) ? 1 : a, cout = (k == L - 1) ? 0 : b;
      int sum = row + cin;
      v = ((sum & 1) == col && (sum >> 1) == cout) ? 1.0 : 0.0;
      break;
    }
  }
  core[t] = v;
}

Tptr mat1d(cudaStream_t s, int kind, int L) {
  int rank = (kind == M_J || kind == M_JT) ? 2 : 1;
  std::vector<int> n(L, 2), m(L, 2), r(L + 1, rank);
  r[0] = r[L] = 1;
  auto t = own(tensor_alloc(L, n.data(), m.data(), r.data(), QTT_F64, 1));
  for (int k = 0; k < L; ++k) {
    mat1d_kernel<<<1, 64, 0, s>>>(kind, k, L, (double*)t->core[k], r[k], r[k + 1]);
    QTT_CHECK_LAUNCH();
  }
  return t;
}

// 1D vector cores (r0, 2, r1) of nodal functions of x = c0 + w i, i = sum 2^(k-1) i_k
enum VecKind { V_ONE = 0, V_LIN = 1, V_SIN = 2, V_COS = 3, V_QUAD = 4, V_E0 = 5, V_EN = 6 };

__global__ void vec1d_kernel(int kind, int k, int L, double c0, double w, double* core, int r0, int r1) {
  int t = threadIdx.x;
  int total = r0 * 2 * r1;
  if (t >= total) return;
  int a = t % r0, i = (t / r0) % 2, b = t / (2 * r0);
  const double wk = w * (double)(1LL << k) * i;   // contribution of this bit
  const bool first = (k == 0), last = (k == L - 1);
  double v = 0.0;
  switch (kind) {
    case V_ONE: v = 1.0; break;
    case V_E0: v = (i == 0); break;
    case V_EN: v = (i == 1); break;
    case V_LIN: {
      // row state (1, s): G = [[1, wk], [0, 1]]
      double G[2][2] = {{1.0, wk}, {0.0, 1.0}};
      if (first && last) v = c0 + wk;
      else if (first) v = (b == 0) ? 1.0 : c0 + wk;
      else if (last) v = (a == 0) ? wk : 1.0;
      else v = G[a][b];
      break;
    }
    case V_QUAD: {
      // row state (1, s, s^2): G = [[1, wk, wk^2], [0, 1, 2 wk], [0, 0, 1]] (i^2 = i)
      double G[3][3] = {{1.0, wk, wk * wk}, {0.0, 1.0, 2.0 * wk}, {0.0, 0.0, 1.0}};
      double s0 = c0 + wk;
      if (first && last) v = s0 * s0;
      else if (first) v = (b == 0) ? 1.0 : (b == 1 ? s0 : s0 * s0);
      else if (last) v = (a == 0) ? wk * wk : (a == 1 ? 2.0 * wk : 1.0);
      else v = G[a][b];
      break;
    }
    case V_SIN:
    case V_COS: {
      // row state (cos theta, sin theta); rotation by phi = wk
      double cph = cos(wk), sph = sin(wk);
      double th = c0 + wk;
      if (first && last) v = (kind == V_SIN) ? sin(th) : cos(th);
      else if (first) v = (b == 0) ? cos(th) : sin(th);
      else if (last) {
        if (kind == V_SIN) v = (a == 0) ? sph : cph;        // [c, s] . [sin phi; cos phi]
        else v = (a == 0) ? cph : -sph;                     // [c, s] . [cos phi; -sin phi]
      } else {
        double R[2][2] = {{cph, sph}, {-sph, cph}};
        v = R[a][b];
      }
      break;
    }
  }
  core[t] = v;
}

Tptr vec1d(cudaStream_t s, int kind, int L, double c0, double w) {
  int rank = 1;
  if (kind == V_LIN || kind == V_SIN || kind == V_COS) rank = 2;
  if (kind == V_QUAD) rank = 3;
  std::vector<int> n(L, 2), r(L + 1, rank);
  r[0] = r[L] = 1;
  auto t = own(tensor_alloc(L, n.data(), nullptr, r.data(), QTT_F64, 0));
  for (int k = 0; k < L; ++k) {
    vec1d_kernel<<<1, 64, 0, s>>>(kind, k, L, c0, w, (double*)t->core[k], r[k], r[k + 1]);
    QTT_CHECK_LAUNCH();
  }
  return t;
}

// ---------------------------------------------------------------------------
// z-kron, Hadamard, diag, transpose kernels
// ---------------------------------------------------------------------------
// Z[(a + ra b), i + 2 j, (i' + 2 j'), (a' + ra' b')] = A[a, i, i', a'] B[b, j, j', b']
// (p = 1 for vectors: no column index)
__global__ void zkron_kernel(const double* A, int ra0, int ra1, const double* B, int rb0, int rb1, int p, double* Z) {
  long long total = (long long)ra0 * rb0 * 4 * (p * p) * ra1 * rb1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long u = t;
    int a = (int)(u % ra0); u /= ra0;
    int b = (int)(u % rb0); u /= rb0;
    int row = (int)(u % 4); u /= 4;
    int col = (int)(u % (p * p)); u /= (p * p);
    int a1 = (int)(u % ra1); u /= ra1;
    int b1 = (int)u;
    int i = row & 1, j = row >> 1;
    int ip = (p == 1) ? 0 : (col & 1), jp = (p == 1) ? 0 : (col >> 1);
    // A core (ra0, 2, p, ra1), B core (rb0, 2, p, rb1)
    double va = A[a + (long long)ra0 * (i + 2 * (ip + (long long)p * a1))];
    double vb = B[b + (long long)rb0 * (j + 2 * (jp + (long long)p * b1))];
    Z[t] = va * vb;
  }
}

// Z[(a + ra b), i, (a' + ra' b')] = X[a, i, a'] Y[b, i, b']  (elementwise product)
__global__ void hadamard_kernel(const double* X, int rx0, int rx1, const double* Y, int ry0, int ry1, int n, double* Z) {
  long long total = (long long)rx0 * ry0 * n * rx1 * ry1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long u = t;
    int a = (int)(u % rx0); u /= rx0;
    int b = (int)(u % ry0); u /= ry0;
    int i = (int)(u % n); u /= n;
    int a1 = (int)(u % rx1); u /= rx1;
    int b1 = (int)u;
    Z[t] = X[a + (long long)rx0 * (i + (long long)n * a1)] * Y[b + (long long)ry0 * (i + (long long)n * b1)];
  }
}

// D[a, i, i', b] = [i == i'] X[a, i, b]
__global__ void diag_kernel(const double* X, int r0, int n, int r1, double* D) {
  long long total = (long long)r0 * n * n * r1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long u = t;
    int a = (int)(u % r0); u /= r0;
    int i = (int)(u % n); u /= n;
    int ip = (int)(u % n); u /= n;
    int b = (int)u;
    D[t] = (i == ip) ? X[a + (long long)r0 * (i + (long long)n * b)] : 0.0;
  }
}

// unit core (1, n, m, 1) with a single 1 at (i, j)
__global__ void unit_core_kernel(double* c, int n, int m, int i, int j) {
  int t = threadIdx.x;
  if (t < n * m) c[t] = (t == i + n * j) ? 1.0 : 0.0;
}

Tptr zkron(cudaStream_t s, const qtt_tensor* A, const qtt_tensor* B) {
  QTT_REQUIRE(A->d == B->d && A->is_matrix == B->is_matrix, "zkron: operands differ");
  const int L = A->d, p = A->is_matrix ? 2 : 1;
  std::vector<int> n(L, 4), m(L, A->is_matrix ? 4 : 1), r(L + 1);
  for (int k = 0; k <= L; ++k) r[k] = A->r[k] * B->r[k];
  auto Z = own(tensor_alloc(L, n.data(), m.data(), r.data(), QTT_F64, A->is_matrix));
  for (int k = 0; k < L; ++k) {
    long long total = (long long)r[k] * 4 * p * p * r[k + 1];
    zkron_kernel<<<grid_for(total), 256, 0, s>>>((const double*)A->core[k], A->r[k], A->r[k + 1],
                                                  (const double*)B->core[k], B->r[k], B->r[k + 1], p,
                                                  (double*)Z->core[k]);
    QTT_CHECK_LAUNCH();
  }
  return Z;
}

Tptr hadamard(cudaStream_t s, const qtt_tensor* X, const qtt_tensor* Y) {
  QTT_REQUIRE(X->d == Y->d && !X->is_matrix && !Y->is_matrix, "hadamard: operands differ");
  const int d = X->d;
  std::vector<int> r(d + 1);
  for (int k = 0; k <= d; ++k) r[k] = X->r[k] * Y->r[k];
  auto Z = own(tensor_alloc(d, X->n, nullptr, r.data(), QTT_F64, 0));
  for (int k = 0; k < d; ++k) {
    long long total = (long long)r[k] * X->n[k] * r[k + 1];
    hadamard_kernel<<<grid_for(total), 256, 0, s>>>((const double*)X->core[k], X->r[k], X->r[k + 1],
                                                     (const double*)Y->core[k], Y->r[k], Y->r[k + 1], X->n[k],
                                                     (double*)Z->core[k]);
    QTT_CHECK_LAUNCH();
  }
  return Z;
}

Tptr diag_of(cudaStream_t s, const qtt_tensor* X) {
  const int d = X->d;
  auto D = own(tensor_alloc(d, X->n, X->n, X->r, QTT_F64, 1));
  for (int k = 0; k < d; ++k) {
    long long total = (long long)X->r[k] * X->n[k] * X->n[k] * X->r[k + 1];
    diag_kernel<<<grid_for(total), 256, 0, s>>>((const double*)X->core[k], X->r[k], X->n[k], X->r[k + 1],
                                                 (double*)D->core[k]);
    QTT_CHECK_LAUNCH();
  }
  return D;
}

Tptr transpose_of(cudaStream_t s, const qtt_tensor* A) {
  const int d = A->d;
  auto T = own(tensor_alloc(d, A->m, A->n, A->r, QTT_F64, 1));
  for (int k = 0; k < d; ++k) {
    int dims[4] = {A->r[k], A->n[k], A->m[k], A->r[k + 1]}, perm[4] = {0, 2, 1, 3};
    permute<double>(s, (const double*)A->core[k], (double*)T->core[k], 4, dims, perm);
  }
  return T;
}

Tptr scaled(cudaStream_t s, const qtt_tensor* X, double a) {
  auto Y = own(tensor_clone(X, QTT_F64, s));
  axpby<double>(s, core_elems(Y.get(), 0), a, (const double*)X->core[0], 0.0, (double*)Y->core[0]);
  return Y;
}

Tptr add(cudaStream_t s, Arena& ar, const qtt_tensor* X, double a, const qtt_tensor* Y, double b, double tol) {
  auto Z = own(tt_sum<double>(s, a, X, b, Y));
  if (tol > 0) round_tt<double>(s, ar, Z.get(), tol, 0);
  return Z;
}

Tptr prod(cudaStream_t s, Arena& ar, const qtt_tensor* A, const qtt_tensor* X, double tol) {
  auto Y = own(product<double>(s, A, X));
  if (tol > 0) round_tt<double>(s, ar, Y.get(), tol, 0);
  return Y;
}

// X (x) unit cores: appends rank-1 cores E_{ij} of sizes (n, m)
Tptr append_units(cudaStream_t s, const qtt_tensor* X, const std::vector<int>& ns, const std::vector<int>& ms,
                  const std::vector<int>& is, const std::vector<int>& js) {
  const int d = X->d, e = (int)ns.size();
  std::vector<int> n(d + e), m(d + e), r(d + e + 1, 1);
  for (int k = 0; k < d; ++k) {
    n[k] = X->n[k];
    m[k] = X->m[k];
    r[k] = X->r[k];
  }
  r[d] = 1;
  for (int k = 0; k < e; ++k) {
    n[d + k] = ns[k];
    m[d + k] = ms[k];
  }
  auto Y = own(tensor_alloc(d + e, n.data(), m.data(), r.data(), QTT_F64, X->is_matrix));
  for (int k = 0; k < d; ++k)
    QTT_CUDA(cudaMemcpyAsync(Y->core[k], X->core[k], core_elems(X, k) * 8, cudaMemcpyDeviceToDevice, s));
  for (int k = 0; k < e; ++k) {
    unit_core_kernel<<<1, 256, 0, s>>>((double*)Y->core[d + k], ns[k], ms[k], is[k], js[k]);
    QTT_CHECK_LAUNCH();
  }
  return Y;
}

// ---------------------------------------------------------------------------
// Geometry (host logic): constrained features of each patch
// ---------------------------------------------------------------------------
struct Feature {
  int kind;   // 0 = side (value = side index), 1 = corner (ci, cj in {0, 1})
  int side, ci, cj;
};

// closed unit segment on the boundary of patch p, side s: endpoints in patch units
void side_segment(const int* xy, int s, int& x0, int& y0, int& x1, int& y1) {
  int ox = xy[0], oy = xy[1];
  switch (s) {
    case 0: x0 = ox; y0 = oy; x1 = ox; y1 = oy + 1; break;            // left
    case 1: x0 = ox + 1; y0 = oy; x1 = ox + 1; y1 = oy + 1; break;    // right
    case 2: x0 = ox; y0 = oy; x1 = ox + 1; y1 = oy; break;            // bottom
    default: x0 = ox; y0 = oy + 1; x1 = ox + 1; y1 = oy + 1; break;   // top
  }
}

// features of patch m lying on patch p's side s (segment intersection)
void intersect_features(const int* xy_m, const int* xy_p, int s, std::vector<Feature>& out) {
  int x0, y0, x1, y1;
  side_segment(xy_p, s, x0, y0, x1, y1);
  int ox = xy_m[0], oy = xy_m[1];
  // each of m's sides: same segment -> whole side
  for (int t = 0; t < 4; ++t) {
    int a0, b0, a1, b1;
    side_segment(xy_m, t, a0, b0, a1, b1);
    if (a0 == x0 && b0 == y0 && a1 == x1 && b1 == y1) {
      out.push_back({0, t, 0, 0});
      return;
    }
  }
  // otherwise corners of m on the segment
  for (int ci = 0; ci < 2; ++ci)
    for (int cj = 0; cj < 2; ++cj) {
      int px = ox + ci, py = oy + cj;
      bool on = (x0 == x1) ? (px == x0 && py >= y0 && py <= y1) : (py == y0 && px >= x0 && px <= x1);
      if (on) out.push_back({1, 0, ci, cj});
    }
}

double gamma_default(int L, double C11, double C33) {
  const double n = (double)(1LL << L), h = 1.0 / (n - 1.0);
  const double trS = (2.0 * n - 2.0) / h, trM = h * (4.0 * n - 4.0) / 6.0;
  return (C11 + C33) * trS * trM / (n * n);
}

}  // namespace

void assemble(const qtt_problem* P, qtt_tensor** Kout, qtt_tensor** fout, cudaStream_t s) {
  QTT_REQUIRE(P && Kout && fout, "qtt_assemble_stiffness: null argument");
  const int L = P->L, q = P->q;
  QTT_REQUIRE(L >= 1 && L <= 18, "qtt_assemble_stiffness: L must be in [1, 18]");
  QTT_REQUIRE(q >= 1 && q <= 16, "qtt_assemble_stiffness: q must be in [1, 16]");
  QTT_REQUIRE(P->patch_xy && P->bc, "qtt_assemble_stiffness: null patch or bc array");
  QTT_REQUIRE(P->E > 0 && P->nu > -1.0 && P->nu < 0.5, "qtt_assemble_stiffness: bad material constants");
  for (int i = 0; i < 4 * q; ++i) QTT_REQUIRE(P->bc[i] >= 0 && P->bc[i] <= 3, "qtt_assemble_stiffness: bad bc flag");
  for (int t = 0; t < P->n_body; ++t) {
    const int* bt = P->body_terms + 3 * t;
    QTT_REQUIRE(bt[0] >= 0 && bt[0] <= 1 && bt[1] >= 0 && bt[1] <= 4 && bt[2] >= 0 && bt[2] <= 4,
                "qtt_assemble_stiffness: bad body-force term");
  }
  for (int t = 0; t < P->n_trac; ++t) {
    const int* tw = P->trac_where + 2 * t;
    QTT_REQUIRE(tw[0] >= 0 && tw[0] < q && tw[1] >= 0 && tw[1] <= 3, "qtt_assemble_stiffness: bad traction");
  }
  QTT_REQUIRE(P->n_dir >= 0 && (P->n_dir == 0 || (P->dir_terms && P->dir_coef)),
              "qtt_assemble_stiffness: bad prescribed-displacement terms");
  for (int t = 0; t < P->n_dir; ++t) {
    const int* dt = P->dir_terms + 3 * t;
    QTT_REQUIRE(dt[0] >= 0 && dt[0] <= 1 && dt[1] >= 0 && dt[1] <= 4 && dt[2] >= 0 && dt[2] <= 4,
                "qtt_assemble_stiffness: bad prescribed-displacement term");
  }
  const double tol = P->tol > 0 ? P->tol : 1e-13;
  const double tin = tol * 1e-2;               // intermediate sums keep more accuracy
  Arena ar(s);
  const double n = (double)(1LL << L), h = 1.0 / (n - 1.0);
  const double e = P->E / (1.0 - P->nu * P->nu);
  const double C11 = e, C22 = e, C12 = e * P->nu, C33 = e * 0.5 * (1.0 - P->nu);
  const double gamma = P->gamma != 0.0 ? P->gamma : gamma_default(L, C11, C33);

  // 1D factors
  auto I1 = mat1d(s, M_I, L), J1 = mat1d(s, M_J, L), JT1 = mat1d(s, M_JT, L);
  auto P0 = mat1d(s, M_P0, L), PN = mat1d(s, M_PN, L);
  auto lin5 = [&](double cI, double cP0, double cPN, double cJ, double cJT) {
    auto acc = scaled(s, I1.get(), cI);
    acc = add(s, ar, acc.get(), 1.0, P0.get(), cP0, 0);
    acc = add(s, ar, acc.get(), 1.0, PN.get(), cPN, 0);
    acc = add(s, ar, acc.get(), 1.0, J1.get(), cJ, 0);
    acc = add(s, ar, acc.get(), 1.0, JT1.get(), cJT, tin);
    return acc;
  };
  auto S1 = lin5(2.0 / h, -1.0 / h, -1.0 / h, -1.0 / h, -1.0 / h);
  auto M1 = lin5(4.0 * h / 6.0, -2.0 * h / 6.0, -2.0 * h / 6.0, h / 6.0, h / 6.0);
  auto G1 = lin5(0.0, -0.5, 0.5, -0.5, 0.5);
  auto G1T = transpose_of(s, G1.get());

  // 2D blocks of one patch: xx, xy, yx, yy
  auto SM = zkron(s, S1.get(), M1.get()), MS = zkron(s, M1.get(), S1.get());
  auto GGt = zkron(s, G1.get(), G1T.get()), GtG = zkron(s, G1T.get(), G1.get());
  Tptr blk[4] = {add(s, ar, SM.get(), C11, MS.get(), C33, tin), add(s, ar, GGt.get(), C12, GtG.get(), C33, tin),
                 add(s, ar, GtG.get(), C12, GGt.get(), C33, tin), add(s, ar, MS.get(), C22, SM.get(), C33, tin)};

  // connectivity Pi^(mp) (z-kron of 1D pieces) for patches at unit offsets
  std::vector<Tptr> Pi;
  std::vector<int> adj(q * q, 0);
  Pi.reserve(q * q);
  for (int a = 0; a < q; ++a)
    for (int b = 0; b < q; ++b) {
      int dx = P->patch_xy[2 * b] - P->patch_xy[2 * a], dy = P->patch_xy[2 * b + 1] - P->patch_xy[2 * a + 1];
      if (a == b || std::max(std::abs(dx), std::abs(dy)) != 1) {
        Pi.push_back(own(nullptr));
        continue;
      }
      auto part = [&](int dd) { return dd == 1 ? mat1d(s, M_E10, L) : (dd == -1 ? mat1d(s, M_E01, L) : mat1d(s, M_I, L)); };
      auto px = part(dx), py = part(dy);
      Pi.push_back(zkron(s, px.get(), py.get()));
      adj[a * q + b] = 1;
    }

  // masks per patch and component: product of (1 - indicator) over features
  auto ones1 = vec1d(s, V_ONE, L, 0, 0), e01 = vec1d(s, V_E0, L, 0, 0), eN1 = vec1d(s, V_EN, L, 0, 0);
  auto ones2 = zkron(s, ones1.get(), ones1.get());
  std::vector<Tptr> mask;  // index m * 2 + c
  for (int m = 0; m < q; ++m) {
    for (int c = 0; c < 2; ++c) {
      std::vector<Feature> feats;
      for (int p = 0; p < q; ++p)
        for (int sd = 0; sd < 4; ++sd)
          if (P->bc[4 * p + sd] & (1 << c)) intersect_features(P->patch_xy + 2 * m, P->patch_xy + 2 * p, sd, feats);
      auto acc = own(tensor_clone(ones2.get(), QTT_F64, s));
      for (const Feature& f : feats) {
        Tptr ind = own(nullptr);
        if (f.kind == 0) {
          if (f.side == 0) ind = zkron(s, e01.get(), ones1.get());
          else if (f.side == 1) ind = zkron(s, eN1.get(), ones1.get());
          else if (f.side == 2) ind = zkron(s, ones1.get(), e01.get());
          else ind = zkron(s, ones1.get(), eN1.get());
        } else {
          ind = zkron(s, f.ci ? eN1.get() : e01.get(), f.cj ? eN1.get() : e01.get());
        }
        auto factor = add(s, ar, ones2.get(), 1.0, ind.get(), -1.0, 0);
        acc = hadamard(s, acc.get(), factor.get());
        round_tt<double>(s, ar, acc.get(), 1e-15, 0);
      }
      mask.push_back(std::move(acc));
    }
  }

  // nodal values at x = o + h i of a separable factor (sin / cos of pi x)
  auto factor1d = [&](int kind, double o) {
    if (kind == V_SIN || kind == V_COS) return vec1d(s, kind, L, M_PI * o, M_PI * h);
    return vec1d(s, kind, L, o, h);
  };
  // lifting of the prescribed displacement: g_{m,c} = (1 - mask_{m,c}) u0_c
  std::vector<Tptr> lift;   // m * 2 + c (null: none)
  for (int m = 0; m < q; ++m)
    for (int c = 0; c < 2; ++c) {
      Tptr acc = own(nullptr);
      for (int t = 0; t < P->n_dir; ++t) {
        if (P->dir_terms[3 * t] != c) continue;
        auto gx = factor1d(P->dir_terms[3 * t + 1], P->patch_xy[2 * m]);
        auto gy = factor1d(P->dir_terms[3 * t + 2], P->patch_xy[2 * m + 1]);
        auto term = scaled(s, zkron(s, gx.get(), gy.get()).get(), P->dir_coef[t]);
        acc = acc ? add(s, ar, acc.get(), 1.0, term.get(), 1.0, tin) : std::move(term);
      }
      if (acc) {
        auto comp = add(s, ar, ones2.get(), 1.0, mask[2 * m + c].get(), -1.0, tin);
        acc = hadamard(s, acc.get(), comp.get());
        round_tt<double>(s, ar, acc.get(), tin, 0);
      }
      lift.push_back(std::move(acc));
    }
  std::vector<Tptr> Klift;   // sum over (p, b) of the unmasked block B_{ab,mp} times g_{p,b}
  for (int i = 0; i < 2 * q; ++i) Klift.push_back(own(nullptr));

  // patch loads f^(m)_c
  std::vector<Tptr> load;   // m * 2 + c
  for (int m = 0; m < q; ++m) {
    const double ox = P->patch_xy[2 * m], oy = P->patch_xy[2 * m + 1];
    Tptr acc[2] = {own(nullptr), own(nullptr)};
    auto accumulate = [&](int c, Tptr term) {
      if (!acc[c]) acc[c] = std::move(term);
      else acc[c] = add(s, ar, acc[c].get(), 1.0, term.get(), 1.0, tin);
    };
    for (int t = 0; t < P->n_body; ++t) {
      const int c = P->body_terms[3 * t], kx = P->body_terms[3 * t + 1], ky = P->body_terms[3 * t + 2];
      const double a = P->body_coef[t];
      auto gx_of = [&](int kind, double o) {
        // nodal values at x = o + h i; sin/cos of pi x
        if (kind == V_SIN || kind == V_COS) return vec1d(s, kind, L, M_PI * o, M_PI * h);
        return vec1d(s, kind, L, o, h);
      };
      auto gx = gx_of(kx, ox), gy = gx_of(ky, oy);
      auto mx = prod(s, ar, M1.get(), gx.get(), tin), my = prod(s, ar, M1.get(), gy.get(), tin);
      auto term = zkron(s, mx.get(), my.get());
      accumulate(c, scaled(s, term.get(), a));
    }
    for (int t = 0; t < P->n_trac; ++t) {
      if (P->trac_where[2 * t] != m) continue;
      const int sd = P->trac_where[2 * t + 1];
      // edge weights: 1D consistent edge mass times ones = h (1 - e0/2 - eN/2)
      auto w = scaled(s, ones1.get(), h);
      w = add(s, ar, w.get(), 1.0, e01.get(), -0.5 * h, 0);
      w = add(s, ar, w.get(), 1.0, eN1.get(), -0.5 * h, tin);
      Tptr vecw = own(nullptr);
      if (sd == 0) vecw = zkron(s, e01.get(), w.get());
      else if (sd == 1) vecw = zkron(s, eN1.get(), w.get());
      else if (sd == 2) vecw = zkron(s, w.get(), e01.get());
      else vecw = zkron(s, w.get(), eN1.get());
      for (int c = 0; c < 2; ++c) {
        double tv = P->trac_val[2 * t + c];
        if (tv != 0.0) accumulate(c, scaled(s, vecw.get(), tv));
      }
    }
    for (int c = 0; c < 2; ++c) {
      if (!acc[c]) acc[c] = scaled(s, ones2.get(), 0.0);
      load.push_back(std::move(acc[c]));
    }
  }

  // global blocks: B_{ab,mp}, masked, attached to patch and component cores
  Tptr K = own(nullptr), f = own(nullptr);
  auto attach_K = [&](Tptr blkmp, int m, int p, int a, int b) {
    std::vector<int> ns, ms, is, js;
    if (q > 1) { ns.push_back(q); ms.push_back(q); is.push_back(m); js.push_back(p); }
    ns.push_back(2); ms.push_back(2); is.push_back(a); js.push_back(b);
    auto full = append_units(s, blkmp.get(), ns, ms, is, js);
    if (!K) K = std::move(full);
    else K = add(s, ar, K.get(), 1.0, full.get(), 1.0, tin);
  };
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const qtt_tensor* Kab = blk[2 * a + b].get();
      for (int m = 0; m < q; ++m)
        for (int p = 0; p < q; ++p) {
          Tptr B = own(nullptr);
          if (m == p) {
            B = own(tensor_clone(Kab, QTT_F64, s));
            if (a == b)
              for (int o = 0; o < q; ++o)
                if (adj[m * q + o]) {
                  auto PiT = transpose_of(s, Pi[m * q + o].get());
                  auto D = prod(s, ar, Pi[m * q + o].get(), PiT.get(), 0);
                  B = add(s, ar, B.get(), 1.0, D.get(), gamma, tin);
                }
          } else if (adj[m * q + p]) {
            B = prod(s, ar, Pi[m * q + p].get(), Kab, tin);
            if (a == b) B = add(s, ar, B.get(), 1.0, Pi[m * q + p].get(), -gamma, tin);
          } else {
            continue;
          }
          if (lift[2 * p + b]) {   // K g with the blocks before the masks
            auto kg = prod(s, ar, B.get(), lift[2 * p + b].get(), tin);
            Klift[2 * m + a] = Klift[2 * m + a] ? add(s, ar, Klift[2 * m + a].get(), 1.0, kg.get(), 1.0, tin)
                                                : std::move(kg);
          }
          // masks: diag(mask_{m,a}) B diag(mask_{p,b}) (+ diag(1 - mask) on the diagonal)
          auto Dl = diag_of(s, mask[2 * m + a].get());
          auto Dr = diag_of(s, mask[2 * p + b].get());
          B = prod(s, ar, Dl.get(), B.get(), tin);
          B = prod(s, ar, B.get(), Dr.get(), tin);
          if (m == p && a == b) {
            auto comp = add(s, ar, ones2.get(), 1.0, mask[2 * m + a].get(), -1.0, tin);
            auto Dc = diag_of(s, comp.get());
            B = add(s, ar, B.get(), 1.0, Dc.get(), 1.0, tin);
          }
          attach_K(std::move(B), m, p, a, b);
        }
    }
  for (int a = 0; a < 2; ++a)
    for (int m = 0; m < q; ++m) {
      auto g = own(tensor_clone(load[2 * m + a].get(), QTT_F64, s));
      for (int p = 0; p < q; ++p)
        if (adj[m * q + p]) {
          auto pf = prod(s, ar, Pi[m * q + p].get(), load[2 * p + a].get(), 0);
          g = add(s, ar, g.get(), 1.0, pf.get(), 1.0, tin);
        }
      if (Klift[2 * m + a]) g = add(s, ar, g.get(), 1.0, Klift[2 * m + a].get(), -1.0, tin);
      g = hadamard(s, g.get(), mask[2 * m + a].get());
      if (lift[2 * m + a]) g = add(s, ar, g.get(), 1.0, lift[2 * m + a].get(), 1.0, tin);
      round_tt<double>(s, ar, g.get(), tin, 0);
      std::vector<int> ns, ms, is, js;
      if (q > 1) { ns.push_back(q); ms.push_back(1); is.push_back(m); js.push_back(0); }
      ns.push_back(2); ms.push_back(1); is.push_back(a); js.push_back(0);
      auto full = append_units(s, g.get(), ns, ms, is, js);
      if (!f) f = std::move(full);
      else f = add(s, ar, f.get(), 1.0, full.get(), 1.0, tin);
    }
  round_tt<double>(s, ar, K.get(), tol, 0);
  round_tt<double>(s, ar, f.get(), tol, 0);
  QTT_CUDA(cudaStreamSynchronize(s));
  // one patch: K = M K0 M + (I - M) with K0 symmetric is symmetric; the
  // concatenated multi-patch system is not (Section 3.6 reading)
  K->sym = (q == 1) ? 1 : 0;
  auto fe = std::make_shared<FeOperator>();
  fe->L = L;
  fe->q = q;
  fe->patch_xy.assign(P->patch_xy, P->patch_xy + 2 * q);
  fe->bc.assign(P->bc, P->bc + 4 * q);
  fe->E = P->E;
  fe->nu = P->nu;
  fe->gamma = gamma;
  K->fe = fe;
  *Kout = K.release();
  *fout = f.release();
}

}  // namespace qtt

extern "C" int qtt_assemble_stiffness(const qtt_problem* p, qtt_tensor** K, qtt_tensor** f, void* stream) {
  try {
    qtt::StreamScope scope_(reinterpret_cast<cudaStream_t>(stream));
    qtt::assemble(p, K, f, reinterpret_cast<cudaStream_t>(stream));
    return QTT_OK;
  } catch (const qtt::QttError& e) {
    qtt::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    qtt::set_last_error(e.what());
    return QTT_EINVAL;
  }
}
