/*
 * qtt.h -- C ABI of the GB300 QTT linear-algebra engine for 2D plane-stress
 * elasticity (low-rank QTT finite elements on Z-ordered Q1 patch meshes).
 *
 * Layout conventions (Section 4 of the paper; readings fixed by this project)
 * ---------------------------------------------------------------------------
 *  - A QTT vector (MPS) with d cores has cores T_k of shape
 *    (r_{k-1}, n_k, r_k), r_0 = r_d = 1.  A QTT matrix (MPO) has cores A_k of
 *    shape (r_{k-1}, n_k, m_k, r_k): row mode i, column mode j, read as the
 *    long index i + n_k j (the paper's remark on MPO cores).
 *  - Every core is stored COLUMN-MAJOR: element (a, i, b) of an MPS core sits
 *    at a + r_{k-1} (i + n_k b); element (a, i, j, b) of an MPO core at
 *    a + r_{k-1} (i + n_k (j + m_k b)).
 *  - The first core carries the least significant index digit (binary
 *    quantisation of Section 4): full[i_1 + n_1 i_2 + n_1 n_2 i_3 + ...] =
 *    T_1[:, i_1, :] T_2[:, i_2, :] ... T_d[:, i_d, :].
 *  - The elasticity layout of a problem with q patches and n = 2^L nodes per
 *    patch side has D = L + [q > 1] + 1 cores: L position cores of mode 4
 *    with mode index i_l + 2 j_l (the Z-order bit pair of level l, Section
 *    3.2), then a patch core of mode q (omitted for q = 1), then a component
 *    core of mode 2 (x, y) -- the block Kronecker assembly of Section 3.7
 *    places the component outermost.
 *
 * Ownership and streams
 * ---------------------
 *  - qtt_tensor objects are opaque, created by the library, hold their cores
 *    in device memory, and are released with qtt_free.
 *  - Entry points are stream-ordered on the cudaStream_t passed as `stream`
 *    (NULL = legacy default stream).  Entry points whose results decide a
 *    rank (rounding, solving) synchronise that stream before returning.
 *  - Caller buffers (`dst` of qtt_to_full, host core arrays) are owned by the
 *    caller and must not be freed before the call's stream work completes.
 *
 * Errors
 * ------
 *  Every function returns QTT_OK (0) or a negative QTT_E* code; nothing is
 *  thrown across the ABI.  qtt_last_error() returns a thread-local message
 *  describing the most recent failure on the calling thread.
 */
#ifndef QTT_H_
#define QTT_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QTT_OK 0
#define QTT_EINVAL (-1)     /* invalid argument (shape, mode size, pointer) */
#define QTT_ENOMEM (-2)     /* device allocation failed */
#define QTT_ECUDA (-3)      /* a CUDA runtime call or kernel launch failed */
#define QTT_ENOCONV (-4)    /* solver stopped at max_sweeps above tolerance */
#define QTT_ETIMEOUT (-5)   /* a bounded device-side wait gave up */
#define QTT_ERANKCAP (-6)   /* a rank would exceed max_rank at tolerance */

#define QTT_F64 0           /* storage and arithmetic in double */
#define QTT_F32 1           /* storage and arithmetic in float */
#define QTT_MIXED 2         /* solve: FP32 inner AMEn + FP64 refinement */

#define QTT_ORDER_Z_BLOCK 0    /* native QTT order: z-ordered position, patch, component */
#define QTT_ORDER_CANONICAL 1  /* per patch, interleaved components 2 (i + n j) + c */

#define QTT_MAX_CORES 40

typedef struct qtt_tensor qtt_tensor;

/* ------------------------------------------------------------------------ */
/* Tensor objects                                                            */
/* ------------------------------------------------------------------------ */

/* Create a tensor from host cores.  d cores; n[k] row mode sizes; m[k] column
 * mode sizes (NULL or all 1 for an MPS); ranks[0..d], ranks[0] = ranks[d] =
 * 1; prec QTT_F64 (cores are double*) or QTT_F32 (float*).  host_cores[k]
 * points to ranks[k] n[k] m[k] ranks[k+1] column-major elements; they are
 * copied, so the caller keeps ownership.  Returns QTT_EINVAL on bad shapes. */
int qtt_tensor_create(int d, const int* n, const int* m, const int* ranks, int prec,
                      const void* const* host_cores, qtt_tensor** out);

/* Query shape: any pointer may be NULL.  n, m have d entries; ranks d + 1. */
int qtt_tensor_info(const qtt_tensor* t, int* d, int* n, int* m, int* ranks, int* prec);

/* Copy the cores back to host buffers host_dst[k] (sized as in create). */
int qtt_tensor_get_cores(const qtt_tensor* t, void* const* host_dst);

/* Device pointer of core k (column-major), for zero-copy access. */
int qtt_tensor_core_ptr(const qtt_tensor* t, int k, void** dev_ptr);

/* Deep copy, optionally converting precision (QTT_F64 / QTT_F32). */
int qtt_tensor_copy(const qtt_tensor* src, int prec, qtt_tensor** out, void* stream);

void qtt_free(qtt_tensor* t);

const char* qtt_last_error(void);

/* ------------------------------------------------------------------------ */
/* Problem description and assembly (Algorithm 1)                           */
/* ------------------------------------------------------------------------ */

typedef struct {
  int L;                     /* levels: n = 2^L nodes per patch side (Section 3.2) */
  int q;                     /* number of unit-square patches (Section 3.1) */
  const int* patch_xy;       /* 2q ints: integer offset (ox, oy) of each patch */
  double E, nu;              /* Young's modulus, Poisson ratio; plane stress (Eq. Cmat) */
  const int* bc;             /* 4q ints: side flags (left, right, bottom, top) per
                                patch; bit 1 = u_x fixed, bit 2 = u_y fixed (Section 3.8) */
  int n_body;                /* separable body-force terms f_c = a g(x) h(y) */
  const int* body_terms;     /* 3 n_body ints: (component, xkind, ykind);
                                kinds 0..4 = 1, t, sin(pi t), cos(pi t), t^2 */
  const double* body_coef;   /* n_body coefficients a */
  int n_trac;                /* constant edge tractions */
  const int* trac_where;     /* 2 n_trac ints: (patch, side) */
  const double* trac_val;    /* 2 n_trac doubles: (t_x, t_y) */
  double gamma;              /* concatenation penalty (Section 3.6); 0 = mean
                                diagonal of K_xx of one patch */
  double tol;                /* relative rounding tolerance of the assembled
                                K and f (0 = 1e-13) */
  int n_dir;                 /* separable terms of the prescribed displacement
                                u0_c = a g(x) h(y) (Algorithm 1's u0; 0 =
                                homogeneous Dirichlet conditions) */
  const int* dir_terms;      /* 3 n_dir ints: (component, xkind, ykind), kinds as
                                for the body force */
  const double* dir_coef;    /* n_dir coefficients a */
} qtt_problem;

/* Assemble the stiffness MPO K and load MPS f of a problem in FP64 on the
 * device (Algorithm 1: 1D factors -> z-kron -> patch concatenation with
 * connectivity Pi^(mp) and penalty gamma -> component blocks -> Dirichlet
 * masks K <- M K M + (I - M), f <- M (f - K g) + g -> rounding, where
 * g = (I - M) u0 lifts the prescribed displacement: the solution equals u0
 * on every constrained DOF).  Patches are unit
 * squares at integer offsets; two patches share an edge or a corner exactly
 * when their offsets differ by one in one or both directions.  Creates *K and
 * *f (caller frees with qtt_free).  Errors: QTT_EINVAL for L < 1, L > 18,
 * q < 1, q > 16, bad flags or kinds. */
int qtt_assemble_stiffness(const qtt_problem* p, qtt_tensor** K, qtt_tensor** f, void* stream);

/* ------------------------------------------------------------------------ */
/* Core operations                                                           */
/* ------------------------------------------------------------------------ */

/* y = A x, MPO times MPS, core by core:
 *   Y_k[(a, g), i, (b, e)] = sum_j A_k[a, i, j, b] X_k[g, j, e]
 * (the paper's "algebraic matrix-vector operations", Section 4).  The output
 * rank index is (a, g) with a fastest.  If tol > 0 the product is rounded to
 * relative accuracy tol (qtt_round), else returned with ranks R_k r_k.
 * A and x must share precision and mode sizes (A's column modes = x's modes).
 * Creates *y. */
int qtt_matvec(const qtt_tensor* A, const qtt_tensor* x, double tol, int max_rank,
               qtt_tensor** y, void* stream);

/* In-place TT rounding (Oseledets 2011, Alg. 2, cited in Section 1): a
 * left-to-right Householder QR sweep, then a right-to-left truncated-SVD
 * sweep; every bond keeps the smallest rank whose discarded singular values
 * have 2-norm <= tol ||x|| / sqrt(d - 1).  Works for MPS and MPO (mode pairs
 * read as one long index).  max_rank <= 0 means unlimited; if the tolerance
 * needs more than max_rank the bond is cut at max_rank and QTT_ERANKCAP is
 * returned (the tensor is still valid).  Synchronises the stream. */
int qtt_round(qtt_tensor* x, double tol, int max_rank, void* stream);

/* z = alpha x + beta y (ranks add; no rounding).  Creates *z. */
int qtt_axpby(double alpha, const qtt_tensor* x, double beta, const qtt_tensor* y,
              qtt_tensor** z, void* stream);

/* Frobenius norm by left orthogonalisation (stable for small differences:
 * the absolute error is of order eps times the norms of the summands).
 * Writes *out on the host; synchronises the stream. */
int qtt_norm(const qtt_tensor* x, double* out, void* stream);

/* Expand an MPS to a full vector (Section 4 entry-wise formula).  dst is a
 * DEVICE pointer with room for n_elems elements of the tensor's precision;
 * n_elems must equal the product of the mode sizes.  ordering:
 *   QTT_ORDER_Z_BLOCK    -- the native QTT index (z-ordered position, then
 *                           patch, then component);
 *   QTT_ORDER_CANONICAL  -- patch-major blocks, inside a patch the DOF pair
 *                           N_ij = (2 L_ij, 2 L_ij + 1) (0-based) with the
 *                           canonical node number L_ij = i + 2^L j (Section 3.2);
 *                           needs the elasticity layout (L, q inferred from
 *                           the cores: L mode-4 cores, optional mode-q core,
 *                           final mode-2 core).
 * For an MPO, n_elems must equal (prod n)(prod m) and only
 * QTT_ORDER_Z_BLOCK is accepted (dense column-major matrix). */
int qtt_to_full(const qtt_tensor* x, void* dst, size_t n_elems, int ordering, void* stream);

/* qtt_to_full for an MPS in QTT_ORDER_Z_BLOCK, computed without taking any
 * device memory at call time.  The paper has no counterpart: this serves
 * callers that must not enter an allocator while they run.  The partial
 * expansions live in one fixed 32 MiB buffer per device that is part of the
 * library image.
 *   dst, n_elems -- as for qtt_to_full (DEVICE pointer, n_elems = prod n).
 *   Returns QTT_EINVAL for an MPO, a size mismatch, or a tensor whose partial
 *   expansions need more than 32 MiB (checked before any launch).
 * The first call on a device looks the buffer up and may load the module:
 * make it, with that device current, before any stream capture.  Calls that
 * overlap in time on one device share the buffer and race: serialise them.
 * The buffer needs no initial contents (each use writes before it reads). */
int qtt_to_full_noalloc(const qtt_tensor* x, void* dst, size_t n_elems, void* stream);

/* Rank-`rank` FP64 approximation r~ of the residual f - K u (K an MPO, u and
 * f MPS, all FP64) by randomized TT rounding, randomize-then-orthogonalize
 * (Al Daas et al., SIAM J. Sci. Comput. 2023), of the structured sum: the
 * cores of K u are never formed.  This is the residual step of the outer
 * refinement in qtt_solve.  r~ is the orthogonal projection of f - K u onto
 * the span of its left-orthonormal factors, so ||f - K u - r~||^2 =
 * ||f - K u||^2 - ||r~||^2; it equals f - K u (up to rounding) when `rank`
 * reaches the ranks of the sum.  `seed` selects the Gaussian sketch;
 * *kept_norm (may be NULL) receives ||r~||.  Creates *r (left-orthonormal
 * cores, the norm in the last).  QTT_EINVAL on shape or precision mismatch. */
int qtt_round_residual(const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f, int rank,
                       unsigned long long seed, double* kept_norm, qtt_tensor** r, void* stream);

/* ------------------------------------------------------------------------ */
/* Solver (AMEn, cited by the paper for K u = f)                             */
/* ------------------------------------------------------------------------ */

typedef struct {
  double tol;             /* target: max local relative residual per sweep (and
                             the FP64 global relative residual for QTT_MIXED) */
  int max_rank;           /* cap on solution ranks (<= 0: 512) */
  int kick_rank;          /* residual-proxy rank rho used for enrichment (<= 0: 4) */
  int max_sweeps;         /* per AMEn run (<= 0: 30) */
  int local_direct_max;   /* local systems up to this size use dense LU (<= 0: 2048) */
  int local_restart;      /* Krylov iterations per cycle of the larger local
                             systems (<= 0: 40; GMRES at most 64, CG at most
                             1000); every cycle starts from an FP64 residual */
  int local_max_cycles;   /* GMRES restart cycles per local solve (<= 0: 8) */
  int precision;          /* QTT_F64, QTT_F32 or QTT_MIXED */
  int refine_max;         /* QTT_F64 / QTT_MIXED: maximum outer refinement steps
                             (0: 6; < 0: none, the sweeps alone decide) */
  double inner_tol;       /* relative tolerance of each refinement's correction
                             solve (<= 0: 1e-3) */
  int verbose;            /* print per-sweep progress to stderr */
  int tensor_cores;       /* QTT_MIXED, FP32 local operator at ranks >= 32:
                             0 = the autotuner chooses per rank bucket between
                             tcgen05 3xTF32 GEMMs (sm_103) and the persistent
                             SIMT CG kernel by their measured time per
                             iteration; > 0 = always tensor cores; < 0 = always
                             SIMT */
} qtt_solve_opts;

typedef struct {
  int status;             /* QTT_OK or the returned error code */
  int sweeps;             /* total AMEn sweeps (all inner solves) */
  int local_solves;       /* local systems solved */
  int local_iters;        /* Krylov iterations over all local solves */
  int max_rank;           /* largest solution rank */
  int refinements;        /* outer refinement steps taken */
  double max_local_res;   /* last sweep's maximum local relative residual */
  double rel_residual;    /* FP64 ||f - K u|| / ||f|| (computed when tol > 0) */
  double erank;           /* effective rank of the solution (Section 4) */
  int checks;             /* FP64 global residual evaluations */
  double check_ms;        /* host wall time of those evaluations */
  double refine_ms;       /* host wall time of the outer refinement steps
                             (residual rounding, correction solve, update) */
} qtt_solve_info;

/* Solve K u = f.  x0: initial guess (NULL = rank-1 constant); z0: initial
 * residual proxy of rank kick_rank (NULL = a fixed deterministic proxy).  One-
 * directional AMEn sweeps: right-orthogonalise x and z, then for every core
 * build the local Galerkin system from the left/right interface tensors,
 * record its relative residual, solve it (dense LU or restarted GMRES), SVD-
 * truncate it at the smallest rank whose local residual stays <= tol /
 * sqrt(D), enrich the basis with the residual projected on the proxy's
 * interfaces, and update the interfaces; stop when the sweep's maximum local
 * residual is <= tol (or, for QTT_F64 / QTT_MIXED, once the FP64 global
 * relative residual is <= tol).  Local systems above local_direct_max use
 * (Jacobi-preconditioned) CG for a symmetric K, restarted GMRES otherwise;
 * with QTT_MIXED their Krylov cycles apply an FP32 copy of the local
 * operator while interfaces, residuals and truncations stay FP64.  With
 * QTT_F64 / QTT_MIXED, sweeps that stall above tol hand over to outer
 * iterative refinement: the residual f - K u is formed in FP64 and
 * compressed -- element by element and TT-SVD-rounded (qtt_residual_fe_tt,
 * rank <= 128) when K comes from qtt_assemble_stiffness and the relative
 * residual is below 1e-9 (or a correction has failed to halve it), where
 * forming it inside the QTT cores loses its low-frequency part to
 * cancellation; otherwise by the QTT matvec with
 * randomized FP64 rounding (qtt_round_residual) -- K d = r is solved the
 * same way to inner_tol, and u <- round(u + d).  QTT_F32 runs everything in
 * FP32 without refinement.  Creates *x; info may be NULL.  Returns
 * QTT_ENOCONV (with *x valid) if max_sweeps / refine_max run out. */
int qtt_solve(const qtt_tensor* K, const qtt_tensor* f, const qtt_tensor* x0,
              const qtt_tensor* z0, const qtt_solve_opts* opts, qtt_tensor** x,
              qtt_solve_info* info, void* stream);

/* Batched solves of count independent problems (uneven levels, patch counts
 * and ranks are fine): K[i] u[i] = f[i] with optional initial guesses x0[i]
 * (x0 NULL or entries NULL = cold start), one options struct for all.  A
 * work queue is drained by nworkers host threads (<= 0: 8), each issuing its
 * solve's kernels on its own stream; `stream` waits for all of them.  Creates
 * x[i]; info (may be NULL) receives one record per problem.  Returns the
 * first error met (the other results stay valid), else QTT_OK; per-problem
 * convergence is in info[i].status. */
int qtt_solve_batched(int count, const qtt_tensor* const* K, const qtt_tensor* const* f,
                      const qtt_tensor* const* x0, const qtt_solve_opts* opts, int nworkers,
                      qtt_tensor** x, qtt_solve_info* info, void* stream);

/* FP64 relative residual ||f - K u|| / ||f||: the product K u is formed
 * exactly in QTT (ranks R r), the sum f - K u expanded to full format (or
 * normed by orthogonalisation when above 2^28 entries), no rounding.  Writes
 * *out on the host; synchronises the stream. */
int qtt_residual(const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f,
                 double* out, void* stream);

/* The same relative residual with K applied as the finite-element operator
 * it was assembled from (Sections 3.4-3.8): u and f are expanded to full
 * format and K u is the Q1 plane-stress stencil of every patch, the
 * concatenation rows of nodes held by several patch copies (summed stiffness
 * rows plus gamma (cnt u_a - sum of the copies' u)) and the Dirichlet masks.
 * Equal to qtt_residual up to the assembly's rounding of K, in O(N r)
 * instead of O(N R r) flops.  K must come from qtt_assemble_stiffness and not
 * have been rounded in place since (else QTT_EINVAL); u, f FP64 MPS.  This is
 * the global residual qtt_solve checks for such K.  Writes *out on the host;
 * synchronises the stream. */
int qtt_residual_fe(const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f,
                    double* out, void* stream);

/* The residual r = f - K u of qtt_residual_fe as a QTT vector: formed
 * element by element in FP64 with the same operator (no QTT arithmetic, so
 * no cancellation between f and K u inside the cores), reordered to QTT
 * order and compressed by a left-to-right TT-SVD (Section 2's rounding
 * applied to a full vector): every unfolding drops a tail
 * <= eps ||r|| / sqrt(d - 1), ranks <= max_rank.  eps in [1e-6, 1) (wide
 * unfoldings go through their Gram matrix, whose small eigenvectors are
 * accurate to ~1e-16 (sigma_1 / sigma_k)^2); max_rank >= 1.  *r is a new
 * FP64 MPS with left-orthonormal cores, owned by the caller (free with
 * qtt_free); *rel (may be NULL) = ||r|| / ||f|| before compression.
 * K must come from qtt_assemble_stiffness (QTT_EINVAL otherwise).  This is
 * the right-hand side of qtt_solve's outer refinement for such K.  Takes
 * device scratch of a few full vectors; synchronises the stream. */
int qtt_residual_fe_tt(const qtt_tensor* K, const qtt_tensor* u, const qtt_tensor* f,
                       double eps, int max_rank, qtt_tensor** r, double* rel, void* stream);

/* y = K x with the assembled operator applied as its finite-element stencil
 * (the operator of qtt_residual_fe, masks and concatenation rows included)
 * to a full vector.  x, y: DEVICE doubles in QTT_ORDER_CANONICAL (patch-major,
 * DOF 2 (i + 2^L j) + c), n_elems = 2 q 4^L, no aliasing; caller-owned.  K
 * must come from qtt_assemble_stiffness (QTT_EINVAL otherwise).  Takes
 * device scratch; stream-ordered (does not synchronise). */
int qtt_fe_apply(const qtt_tensor* K, const void* x, void* y, size_t n_elems, void* stream);

/* ------------------------------------------------------------------------ */
/* Learned warm start (growth pattern of this engine; not in the paper)      */
/* ------------------------------------------------------------------------ */
/* A 3-layer MLP maps nin load/material features to the cores of a rank-r QTT
 * that seeds qtt_solve.  All arrays are DEVICE float32, column-major, with
 * the batch as the slowest index: phi (nin x B), h1, h2 (H x B), out (P x B),
 * W1 (H x nin), W2 (H x H), W3 (P x H), biases of the layer widths.
 *   h1 = tanh(W1 phi + b1), h2 = tanh(W2 h1 + b2), out = W3 h2 + b3.
 * Core k of sample b is the next r_{k-1} n_k r_k entries of out[:, b]
 * (column-major (r_{k-1}, n_k, r_k), r_0 = r_d = 1). */
int qtt_ws_forward(int B, int nin, int H, int P, const float* W1, const float* b1, const float* W2,
                   const float* b2, const float* W3, const float* b3, const float* phi,
                   float* h1, float* h2, float* out, void* stream);

/* Gradients of the MLP parameters given dLoss/dout (P x B); work is device
 * scratch of 2 H B floats owned by the caller. */
int qtt_ws_backward(int B, int nin, int H, int P, const float* W2, const float* W3, const float* phi,
                    const float* h1, const float* h2, const float* gout, float* gW1, float* gb1,
                    float* gW2, float* gb2, float* gW3, float* gb3, float* work, void* stream);

/* Host Gram matrix gram[t nbasis + u] = <basis_t, basis_u> of FP32 basis
 * tensors (TT inner products; synchronises the stream). */
int qtt_ws_basis_gram(int d, int nbasis, const qtt_tensor* const* basis, double* gram, void* stream);

/* Gauge-invariant loss of each sample, loss[b] = ||X_hat_b - X_b||^2 /
 * ||X_b||^2, with X_hat_b the predicted TT and the target
 * X_b = sum_t coef[b nbasis + t] basis[t] (host coef; FP32 basis tensors of
 * the same modes), computed from TT inner products (transfer matrices).
 * gram: host Gram matrix of the basis from qtt_ws_basis_gram, or NULL to
 * compute it here.  Writes loss (device, B) and gout = d(mean loss)/d(out)
 * (device, P x B). */
int qtt_ws_tt_loss(int B, int d, const int* modes, int r, const float* out, int nbasis,
                   const qtt_tensor* const* basis, const double* coef, const double* gram, float* loss,
                   float* gout, void* stream);

/* One Adam step on n parameters (device arrays; t >= 1 is the step number). */
int qtt_ws_adam(int n, float* w, const float* g, float* m, float* v, float lr, float b1, float b2,
                float eps, int t, void* stream);

/* New FP64 qtt_tensor from one predicted output column (device), the first
 * core multiplied by scale. */
int qtt_ws_to_tensor(const float* out_row, int d, const int* modes, int r, double scale,
                     qtt_tensor** x, void* stream);

/* ------------------------------------------------------------------------ */
/* Dense building block                                                      */
/* ------------------------------------------------------------------------ */

/* D = A B^T in FP32 accuracy on the tcgen05 tensor cores (3xTF32: every
 * operand split into a TF32 pair hi + lo, products hi hi + hi lo + lo hi
 * accumulated in FP32; the dense contractions of the FP32 local operator use
 * the same kernel).  A: M x K, element (m, k) at A[m lda + k]; B: N x K, element
 * (n, k) at B[n ldb + k]; D: M x N column-major, D[m + n ldd].  All DEVICE
 * float pointers owned by the caller; the call takes device scratch for the
 * split operands and synchronises the stream.  When the output tiles cannot
 * fill the SMs the K loop is split over CTAs and accumulated atomically into
 * D (zeroed first), so the summation order is not fixed.  QTT_EINVAL on bad sizes or a
 * device other than sm_103; QTT_ETIMEOUT if a bounded wait in the kernel gave
 * up (the context stays usable). */
int qtt_gemm_tf32x3(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* D, int ldd,
                    void* stream);

/* ------------------------------------------------------------------------ */
/* Diagnostics (not part of the method)                                      */
/* ------------------------------------------------------------------------ */

/* The autotuner's table for the current device: for every rank bucket of
 * the FP32 local operator met so far (b = floor(2 log2 r) for the left and
 * right ranks), the measured microseconds per Krylov iteration on the
 * tensor cores (us_tc) and in the persistent SIMT kernel (us_simt), -1 while
 * not yet timed; later local solves in a bucket take the faster path.  Fills
 * up to cap entries of each (non-NULL) array; *count = entries in the table. */
int qtt_autotune_table(int cap, int* count, int* r0_bucket, int* r1_bucket, double* us_tc, double* us_simt);

/* Number of CUDA kernels this library has launched in this process. */
unsigned long long qtt_kernel_launches(void);

/* Number of device allocations (stream-ordered or not) this library has
 * made in this process. */
unsigned long long qtt_device_allocations(void);

/* Rate of this GPU's FMA pipe in precision prec (QTT_F64 or QTT_F32), in
 * TFLOP/s (one FMA = 2 flops): eight independent FMA chains per thread in 8
 * blocks of 256 threads per SM, timed with CUDA events on `stream` (the
 * second of two launches).  The roofline denominator of the ALU-bound
 * kernels; allocates and frees a small device buffer; synchronises. */
int qtt_measure_fma_peak(int prec, double* tflops, void* stream);

/* on != 0: bracket every launch of the profiled kernel classes with CUDA
 * events on its stream and record its algorithmic flops and bytes (adds
 * launch overhead; off by default).  Classes: 0 FP64 GEMM, 1 FP32 GEMM,
 * 2 MPO x MPS core product, 3 Householder panel, 4 Jacobi SVD, 5 LU panel,
 * 6 permutation, 7 full expansion, 8 persistent FP32 local CG (one launch runs
 * all iterations of a CG cycle), 9 FP32 Jacobi sweeps of the mixed-precision
 * SVD (class 4 then holds the FP64 sweeps), 10 tensor-core 3xTF32 GEMM. */
int qtt_profile_enable(int on);

/* Sum of event-timed milliseconds, algorithmic flops and bytes, and launch
 * count of class cls (-1: all classes) recorded since the last read; waits
 * for the recorded events and clears them. */
int qtt_profile_read(int cls, double* ms, double* flops, double* bytes, long long* launches);

#ifdef __cplusplus
}
#endif

#endif  /* QTT_H_ */
