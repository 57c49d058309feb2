"""O-2: dense-reference tensor-train layer (oracle; test infrastructure only).

Definitions of Section 4:
  * MPS (TT vector) cores T_l of shape (r_{l-1}, n_l, r_l), r_0 = r_d = 1;
    T(i_1..i_d) = T_1[:, i_1, :] T_2[:, i_2, :] ... T_d[:, i_d, :].
  * MPO (TT matrix) cores A_l of shape (r_{l-1}, n_l, m_l, r_l), mode pair
    (i, j) read as the long index i + n j (Remark after the MPO definition).
  * Flattening: the first core carries the least significant index (binary
    quantisation of an index with i_1 the least significant digit), so a full
    vector v satisfies v[i_1 + n_1 i_2 + n_1 n_2 i_3 + ...] = T(i_1, ..., i_d).
Algorithms cited by the paper and restated here from their definitions:
  * TT-SVD, sequential truncated SVDs of the unfoldings (Oseledets 2011,
    Alg. 1), truncation threshold delta = eps ||A||_F / sqrt(d - 1);
  * TT rounding (Oseledets 2011, Alg. 2): an orthogonalising QR sweep
    followed by a truncated-SVD sweep with the same per-bond threshold;
  * the MPO x MPS product, core by core:
      Y_l[(a, g), i, (b, e)] = sum_j A_l[a, i, j, b] X_l[g, j, e];
  * z-kron (Section 3.8 and Section 4): for 1D QTT matrices A (x) and B (y)
    with 2x2 mode cores, (A zkron B)_l[(a, b), i + 2 j, i' + 2 j', (a', b')]
    = A_l[a, i, i', a'] B_l[b, j, j', b'].
  * effective rank and the parameter counts R_d, N_d (Section 4).
Everything is plain NumPy in FP64, no blocking or fusion.
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

Cores = List[np.ndarray]


# ----------------------------------------------------------------------------
# Expansion to full format
# ----------------------------------------------------------------------------

def full(cores: Cores) -> np.ndarray:
    """Full vector of an MPS (first core = least significant index)."""
    acc = cores[0][0]                                   # (n1, r1)
    for G in cores[1:]:
        r0, n, r1 = G.shape
        # acc[(i_1..i_{l-1}), r] -> acc[(i_1..i_l), r'] with i_l the new slowest index
        acc = np.einsum("pr,rns->nps", acc, G).reshape(n * acc.shape[0], r1)
    return acc[:, 0]


def full_matrix(cores: Cores) -> np.ndarray:
    """Dense matrix of an MPO: A[row, col] with row = sum i_l N_{<l},
    col = sum j_l M_{<l}."""
    acc = cores[0][0]                                   # (n1, m1, r1)
    for G in cores[1:]:
        r0, n, m, r1 = G.shape
        N0, M0 = acc.shape[0], acc.shape[1]
        acc = np.einsum("pqr,rnms->npmqs", acc, G).reshape(n * N0, m * M0, r1)
    return acc[:, :, 0]


def ranks(cores: Cores) -> List[int]:
    return [cores[0].shape[0]] + [G.shape[-1] for G in cores]


def modes(cores: Cores) -> List[int]:
    return [G.shape[1] for G in cores]


# ----------------------------------------------------------------------------
# TT-SVD (Oseledets 2011, Alg. 1)
# ----------------------------------------------------------------------------

def _trunc_rank(s: np.ndarray, delta: float) -> int:
    """Smallest rank whose discarded singular-value tail has 2-norm <= delta."""
    tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]   # tail[k] = ||s[k:]||
    keep = len(s)
    for k in range(len(s)):
        if tail[k] <= delta:
            keep = k
            break
    return max(keep, 1)


def tt_svd(v: np.ndarray, mode_sizes: Sequence[int], eps: float, max_rank: int = 1 << 30) -> Cores:
    """TT decomposition of a full vector with relative accuracy eps."""
    d = len(mode_sizes)
    v = np.asarray(v, dtype=np.float64)
    nrm = np.linalg.norm(v)
    delta = eps * nrm / math.sqrt(max(d - 1, 1))
    # column-major flattening: the first mode is the fastest index
    C = v.reshape(list(mode_sizes)[::-1]).transpose(list(range(d))[::-1]).copy()
    cores = []
    r = 1
    rest = C.reshape(r * mode_sizes[0], -1, order="F")
    for k in range(d - 1):
        n = mode_sizes[k]
        rest = rest.reshape(r * n, -1, order="F")
        U, s, Vt = np.linalg.svd(rest, full_matrices=False)
        rk = min(_trunc_rank(s, delta), max_rank)
        cores.append(U[:, :rk].reshape(r, n, rk, order="F"))
        rest = (s[:rk, None] * Vt[:rk])                  # (rk, n_{k+1} ... n_d)
        r = rk
    cores.append(rest.reshape(r, mode_sizes[-1], 1, order="F"))
    return cores


def mpo_from_matrix(A: np.ndarray, rows: Sequence[int], cols: Sequence[int], eps: float = 1e-14) -> Cores:
    """TT-SVD of a dense matrix into MPO cores with mode pairs (rows[l], cols[l])."""
    d = len(rows)
    # C-order axes of the reshaped matrix: (i_d .. i_1, j_d .. j_1)
    T = A.reshape(list(rows)[::-1] + list(cols)[::-1])
    # reorder to (j_d, i_d, ..., j_1, i_1): flattening then gives the long
    # per-level index i_l + n_l j_l with the first level fastest
    ax = []
    for l in range(d, 0, -1):
        ax += [2 * d - l, d - l]
    vec = T.transpose(ax).reshape(-1)
    pair = [rows[l] * cols[l] for l in range(d)]
    cores = tt_svd(vec, pair, eps)
    return [G.reshape(G.shape[0], rows[l], cols[l], G.shape[2], order="F") for l, G in enumerate(cores)]


# ----------------------------------------------------------------------------
# Algebra
# ----------------------------------------------------------------------------

def add(x: Cores, y: Cores) -> Cores:
    """x + y by block-diagonal core concatenation (ranks add)."""
    d = len(x)
    out = []
    for k in range(d):
        a, b = x[k], y[k]
        if d == 1:
            out.append(a + b)
            continue
        sh = list(a.shape)
        if k == 0:
            out.append(np.concatenate([a, b], axis=-1))
        elif k == d - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            sh[0] = a.shape[0] + b.shape[0]
            sh[-1] = a.shape[-1] + b.shape[-1]
            G = np.zeros(sh)
            G[: a.shape[0], ..., : a.shape[-1]] = a
            G[a.shape[0]:, ..., a.shape[-1]:] = b
            out.append(G)
    return out


def scale(x: Cores, alpha: float) -> Cores:
    out = [G.copy() for G in x]
    out[0] = out[0] * alpha
    return out


def kron(x: Cores, y: Cores) -> Cores:
    """Tensor whose first cores are x and last cores are y (x indexes the
    less significant digits): v[i_x + N_x i_y] = x[i_x] y[i_y]."""
    return [G.copy() for G in x] + [G.copy() for G in y]


def matvec(A: Cores, x: Cores) -> Cores:
    """MPO x MPS, core by core: Y[(a,g), i, (b,e)] = sum_j A[a,i,j,b] X[g,j,e]."""
    out = []
    for Ak, Xk in zip(A, x):
        Ra, n, m, Rb = Ak.shape
        ra, m2, rb = Xk.shape
        assert m == m2
        Y = np.einsum("aijb,gje->agibe", Ak, Xk).reshape(Ra * ra, n, Rb * rb)
        out.append(Y)
    return out


def matmat(A: Cores, B: Cores) -> Cores:
    """MPO x MPO: C[(a,g), i, k, (b,e)] = sum_j A[a,i,j,b] B[g,j,k,e]."""
    out = []
    for Ak, Bk in zip(A, B):
        Ra, n, m, Rb = Ak.shape
        ra, m2, p, rb = Bk.shape
        out.append(np.einsum("aijb,gjke->agikbe", Ak, Bk).reshape(Ra * ra, n, p, Rb * rb))
    return out


def diag_mpo(x: Cores) -> Cores:
    """MPO of diag(x)."""
    out = []
    for G in x:
        r0, n, r1 = G.shape
        D = np.zeros((r0, n, n, r1))
        for i in range(n):
            D[:, i, i, :] = G[:, i, :]
        out.append(D)
    return out


def identity_mpo(mode_sizes: Sequence[int]) -> Cores:
    return [np.eye(n).reshape(1, n, n, 1) for n in mode_sizes]


def transpose_mpo(A: Cores) -> Cores:
    return [G.transpose(0, 2, 1, 3).copy() for G in A]


def zkron(A: Cores, B: Cores) -> Cores:
    """z-kron of two 1D QTT matrices with 2x2 mode cores (A acts on the x bit
    i, B on the y bit j): mode index i + 2 j at every level."""
    out = []
    for Ak, Bk in zip(A, B):
        ra, n1, m1, ra2 = Ak.shape
        rb, n2, m2, rb2 = Bk.shape
        # C[(a,b), i, j, i', j', (a',b')] -> long row i + n1 j, long col i' + m1 j'
        C = np.einsum("aipc,bjqd->abjiqpcd", Ak, Bk)      # a, b, j, i, q(j'), p(i'), c, d
        C = C.reshape(ra * rb, n2, n1, m2, m1, ra2 * rb2)
        # row long index i + n1 j: reshape (n2, n1) with i fastest -> order (j, i) C-order = i + n1 j
        C = C.reshape(ra * rb, n1 * n2, m1 * m2, ra2 * rb2)
        out.append(C)
    return out


def zkron_vec(a: Cores, b: Cores) -> Cores:
    """z-kron of two 1D QTT vectors (mode-2 cores): mode index i + 2 j."""
    out = []
    for Ak, Bk in zip(a, b):
        ra, n1, ra2 = Ak.shape
        rb, n2, rb2 = Bk.shape
        C = np.einsum("aic,bjd->abjicd", Ak, Bk).reshape(ra * rb, n1 * n2, ra2 * rb2)
        out.append(C)
    return out


# ----------------------------------------------------------------------------
# Orthogonalisation, norms, rounding (Oseledets 2011, Alg. 2)
# ----------------------------------------------------------------------------

def _as_mps(x: Cores):
    """View MPO cores as MPS cores with long mode index (i + n j)."""
    shapes = [G.shape for G in x]
    if x[0].ndim == 4:
        return [G.reshape(G.shape[0], G.shape[1] * G.shape[2], G.shape[3], order="F") for G in x], shapes
    return [G.copy() for G in x], shapes


def _from_mps(x: Cores, shapes) -> Cores:
    if len(shapes[0]) == 4:
        return [G.reshape(G.shape[0], s[1], s[2], G.shape[2], order="F") for G, s in zip(x, shapes)]
    return x


def left_orthogonalize(x: Cores, upto: int = None) -> Cores:
    """QR sweep left to right: cores 0..upto-1 become left-orthonormal."""
    y, shapes = _as_mps(x)
    d = len(y)
    upto = d - 1 if upto is None else upto
    for k in range(upto):
        r0, n, r1 = y[k].shape
        Q, R = np.linalg.qr(y[k].reshape(r0 * n, r1, order="F"))
        y[k] = Q.reshape(r0, n, Q.shape[1], order="F")
        y[k + 1] = np.einsum("ab,bnc->anc", R, y[k + 1])
    return _from_mps(y, shapes)


def right_orthogonalize(x: Cores, downto: int = 0) -> Cores:
    """QR sweep right to left: cores downto+1..d-1 become right-orthonormal."""
    y, shapes = _as_mps(x)
    d = len(y)
    for k in range(d - 1, downto, -1):
        r0, n, r1 = y[k].shape
        Q, R = np.linalg.qr(y[k].reshape(r0, n * r1, order="F").T)
        y[k] = Q.T.reshape(Q.shape[1], n, r1, order="F")
        y[k - 1] = np.einsum("anb,cb->anc", y[k - 1], R)
    return _from_mps(y, shapes)


def norm(x: Cores) -> float:
    """Frobenius norm via left orthogonalisation (stable for differences)."""
    y = left_orthogonalize(x)
    return float(np.linalg.norm(y[-1]))


def dot(x: Cores, y: Cores) -> float:
    """<x, y> by the left transfer contraction."""
    xm, _ = _as_mps(x)
    ym, _ = _as_mps(y)
    P = np.ones((1, 1))
    for X, Y in zip(xm, ym):
        P = np.einsum("ab,anc,bnd->cd", P, X, Y)
    return float(P[0, 0])


def round_tt(x: Cores, eps: float, max_rank: int = 1 << 30) -> Cores:
    """TT rounding: left-to-right QR sweep, then right-to-left truncated SVD
    sweep; per-bond threshold delta = eps ||x|| / sqrt(d - 1); a bond keeps
    the smallest rank whose discarded tail is <= delta."""
    y, shapes = _as_mps(x)
    d = len(y)
    if d == 1:
        return _from_mps(y, shapes)
    y = left_orthogonalize(y)
    nrm = np.linalg.norm(y[-1])
    delta = eps * nrm / math.sqrt(d - 1)
    for k in range(d - 1, 0, -1):
        r0, n, r1 = y[k].shape
        U, s, Vt = np.linalg.svd(y[k].reshape(r0, n * r1, order="F"), full_matrices=False)
        rk = min(_trunc_rank(s, delta), max_rank)
        y[k] = Vt[:rk].reshape(rk, n, r1, order="F")
        y[k - 1] = np.einsum("anb,bc->anc", y[k - 1], U[:, :rk] * s[:rk])
    return _from_mps(y, shapes)


# ----------------------------------------------------------------------------
# Reporting quantities (Section 4)
# ----------------------------------------------------------------------------

def storage(x: Cores) -> int:
    return int(sum(G.size for G in x))


def erank(x: Cores) -> float:
    """Effective rank r_e: r_e n_1 + sum_{i=2}^{d-1} r_e^2 n_i + r_e n_d =
    storage, solved for the positive root (mode size n_i counts all mode
    indices of core i)."""
    n = [int(np.prod(G.shape[1:-1])) for G in x]
    S = storage(x)
    if len(x) == 1:
        return 1.0
    a = float(sum(n[1:-1]))
    b = float(n[0] + n[-1])
    if a == 0.0:
        return S / b
    return (-b + math.sqrt(b * b + 4 * a * S)) / (2 * a)


def max_rank(x: Cores) -> int:
    """R_d = max_i r_i (Eq. Rd)."""
    return int(max(ranks(x)))


def n_params(x: Cores) -> int:
    """N_d = number of stored parameters (Eq. Nd counts the core entries)."""
    return storage(x)
