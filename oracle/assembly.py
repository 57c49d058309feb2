"""O-2: QTT assembly of K and f (Algorithm 1; oracle, test infrastructure).

The steps follow Algorithm 1 and Sections 3.5-3.8:
  * element integrals K_(c1,c2) and G_(c1,c2) by the 2x2 Gauss rule (taken
    from the O-1 element routines);
  * shift matrices V_c moving element values to corner c's node; with
    elements indexed like their bottom-left node, V_c1^T diag(k) V_c2
    separates into a z-kron of 1D factors
        T(a, b)[i, i'] = sum_e [i = e + a] valid(e) [i' = e + b],
    valid(e) = 1 for e <= n - 2 (Eq. Nodal:Stiffness:Matrix);
  * K^(m) = sum over the sixteen corner pairs (Eq. Subdomain:Stiffness:
    Matrix); f^(m) = sum of V^T diag(G) V fbar (Eq. load:vector:intensity);
  * concatenation with connectivity matrices Pi^(mp) and penalty gamma
    (Section 3.6, read as: diagonal blocks K^(m) + gamma D_m, off-diagonal
    blocks Pi^(mp) K^(p) - gamma Pi^(mp), gamma only on the xx and yy
    blocks; g_m = f_m + sum_p Pi^(mp) f_p);
  * block Kronecker assembly over components (Section 3.7) with the
    component index outermost;
  * homogeneous Dirichlet masks (Section 3.8), applied as
    K <- M K M + (I - M), f <- M f.
The 1D factors are obtained by TT-SVD of their dense n x n matrices, so this
route shares nothing with a closed-form construction.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

from . import fem, tt

Cores = List[np.ndarray]
EPS_EXACT = 1e-14


# ----------------------------------------------------------------------------
# 1D factors (dense -> TT-SVD)
# ----------------------------------------------------------------------------

def shift_product_dense(n: int, a: int, b: int) -> np.ndarray:
    """T(a, b) = V_a^T diag(valid) V_b for one direction (dense, n x n)."""
    T = np.zeros((n, n))
    for e in range(n - 1):
        T[e + a, e + b] += 1.0
    return T


def qtt_matrix_1d(Md: np.ndarray, L: int) -> Cores:
    return tt.mpo_from_matrix(Md, [2] * L, [2] * L, EPS_EXACT)


def qtt_vector_1d(v: np.ndarray, L: int) -> Cores:
    return tt.tt_svd(v, [2] * L, EPS_EXACT)


# ----------------------------------------------------------------------------
# Patch stiffness blocks and loads in QTT (z-ordered)
# ----------------------------------------------------------------------------

# corner c of Section 3.4 -> (cx, cy) offset of its node within the element
_CORNER_OFFSETS = [(0, 0), (1, 0), (1, 1), (0, 1)]


def patch_blocks(L: int, E: float, nu: float, eps: float = 1e-13):
    """K^(m)_{ab}, a, b in {x, y}, as z-ordered QTT matrices (4 lists of cores
    in the order xx, xy, yx, yy)."""
    n = 1 << L
    h = 1.0 / (n - 1)
    C = fem.plane_stress_C(E, nu)
    Ke = fem.element_stiffness(np.array([[0, 0], [h, 0], [h, h], [0, h]], dtype=float), C)
    T1 = {(a, b): qtt_matrix_1d(shift_product_dense(n, a, b), L) for a in (0, 1) for b in (0, 1)}
    blocks = []
    for alpha in (0, 1):
        for beta in (0, 1):
            acc = None
            for c1, (ax, ay) in enumerate(_CORNER_OFFSETS):
                for c2, (bx, by) in enumerate(_CORNER_OFFSETS):
                    k = Ke[2 * c1 + alpha, 2 * c2 + beta]
                    if k == 0.0:
                        continue
                    term = tt.scale(tt.zkron(T1[(ax, bx)], T1[(ay, by)]), k)
                    acc = term if acc is None else tt.round_tt(tt.add(acc, term), eps * 1e-3)
            blocks.append(tt.round_tt(acc, eps))
    return blocks


def _edge_vector(n: int, side_end: int) -> np.ndarray:
    v = np.zeros(n)
    v[0 if side_end == 0 else n - 1] = 1.0
    return v


def patch_load_qtt(prob, m: int, eps: float = 1e-13):
    """(f_x, f_y) of patch m as z-ordered QTT vectors."""
    L, n = prob.L, prob.n
    h = 1.0 / (n - 1)
    ox, oy = prob.patches[m]
    xs = ox + h * np.arange(n)
    ys = oy + h * np.arange(n)
    Me = fem.element_mass(np.array([[0, 0], [h, 0], [h, h], [0, h]], dtype=float))
    T1 = {(a, b): qtt_matrix_1d(shift_product_dense(n, a, b), L) for a in (0, 1) for b in (0, 1)}
    out = [None, None]
    for comp, coeff, kx, ky in prob.body:
        gx = qtt_vector_1d(fem._body_factor(kx, xs), L)
        gy = qtt_vector_1d(fem._body_factor(ky, ys), L)
        fbar = tt.scale(tt.zkron_vec(gx, gy), coeff)
        for c1, (ax, ay) in enumerate(_CORNER_OFFSETS):
            for c2, (bx, by) in enumerate(_CORNER_OFFSETS):
                V = tt.zkron(T1[(ax, bx)], T1[(ay, by)])
                term = tt.scale(tt.matvec(V, fbar), Me[c1, c2])
                out[comp] = term if out[comp] is None else tt.round_tt(tt.add(out[comp], term), eps * 1e-3)
    # traction: 1D consistent edge mass x nodal traction on the side
    Me1 = fem.edge_mass(h)
    wdense = np.zeros(n)
    for e in range(n - 1):
        wdense[e:e + 2] += Me1 @ np.ones(2)
    for (pm, side, tx, ty) in prob.traction:
        if pm != m:
            continue
        w = qtt_vector_1d(wdense, L)
        if side in (0, 1):       # left/right: constant i, varying j
            sel = qtt_vector_1d(_edge_vector(n, side), L)
            vec = tt.zkron_vec(sel, w)
        else:                    # bottom/top: varying i, constant j
            sel = qtt_vector_1d(_edge_vector(n, side - 2), L)
            vec = tt.zkron_vec(w, sel)
        for comp, t in ((0, tx), (1, ty)):
            if t == 0.0:
                continue
            term = tt.scale(vec, t)
            out[comp] = term if out[comp] is None else tt.round_tt(tt.add(out[comp], term), eps * 1e-3)
    for comp in (0, 1):
        if out[comp] is None:
            out[comp] = [np.zeros((1, 4, 1)) for _ in range(L)]
        else:
            out[comp] = tt.round_tt(out[comp], eps)
    return out


# ----------------------------------------------------------------------------
# Connectivity, masks, global assembly
# ----------------------------------------------------------------------------

def _edge_selector(n: int, a: int, b: int) -> np.ndarray:
    M = np.zeros((n, n))
    M[a, b] = 1.0
    return M


def connectivity(prob, m: int, p: int):
    """Pi^(mp) as a z-ordered QTT matrix, or None if the patches share no
    node.  Patches are unit squares at integer offsets, so the shared set is
    an edge (offset difference one in one direction) or a corner."""
    n, L = prob.n, prob.L
    dx = prob.patches[p][0] - prob.patches[m][0]
    dy = prob.patches[p][1] - prob.patches[m][1]
    if max(abs(dx), abs(dy)) != 1:
        return None

    def part(d):
        if d == 1:
            return _edge_selector(n, n - 1, 0)    # m's last node meets p's first
        if d == -1:
            return _edge_selector(n, 0, n - 1)
        return np.eye(n)

    return tt.zkron(qtt_matrix_1d(part(dx), L), qtt_matrix_1d(part(dy), L))


def mask_qtt(prob, eps: float = 1e-14) -> Cores:
    """Global 0/1 mask over the QTT layout (1 = free DOF), from the node
    flags of every patch compressed by TT-SVD."""
    L, q, n = prob.L, prob.q, prob.n
    flags = fem.constrained_flags(prob)
    from .indexing import zorder
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    z = zorder(ii, jj, L).ravel()
    nn = n * n
    full = np.ones(2 * q * nn)
    for m in range(q):
        fl = flags[m].ravel()
        for c, bit in ((0, 1), (1, 2)):
            full[z[(fl & bit) != 0] + nn * m + nn * q * c] = 0.0
    modes = [4] * L + ([q] if q > 1 else []) + [2]
    return tt.tt_svd(full, modes, eps)


def _unit(n: int, i: int) -> np.ndarray:
    v = np.zeros(n)
    v[i] = 1.0
    return v


def _unit_matrix(n: int, i: int, j: int) -> np.ndarray:
    M = np.zeros((n, n))
    M[i, j] = 1.0
    return M


def gamma_default(prob) -> float:
    """Mean diagonal of K^(m)_xx (Section 3.6)."""
    return fem.mean_diag_Kxx(prob)


def assemble(prob, eps: float = 1e-13):
    """Algorithm 1: returns (K MPO cores, f MPS cores) in the QTT layout
    (L position cores, patch core if q > 1, component core)."""
    L, q = prob.L, prob.q
    blocks = patch_blocks(L, prob.E, prob.nu, eps)          # xx, xy, yx, yy
    gamma = prob.gamma if prob.gamma != 0.0 else gamma_default(prob)
    loads = [patch_load_qtt(prob, m, eps) for m in range(q)]
    Pi = {(m, p): connectivity(prob, m, p) for m in range(q) for p in range(q) if m != p}

    def attach_matrix(pos: Cores, mp, ab) -> Cores:
        tail = []
        if q > 1:
            tail.append(_unit_matrix(q, *mp).reshape(1, q, q, 1))
        tail.append(_unit_matrix(2, *ab).reshape(1, 2, 2, 1))
        return tt.kron(pos, tail)

    def attach_vector(pos: Cores, m, a) -> Cores:
        tail = []
        if q > 1:
            tail.append(_unit(q, m).reshape(1, q, 1))
        tail.append(_unit(2, a).reshape(1, 2, 1))
        return tt.kron(pos, tail)

    K = None
    f = None

    def acc_add(acc, term):
        return term if acc is None else tt.round_tt(tt.add(acc, term), eps * 1e-2)

    for ia, a in enumerate((0, 1)):
        for ib, b in enumerate((0, 1)):
            Kab = blocks[2 * a + b]
            for m in range(q):
                # diagonal block K^(m) + gamma D_m (xx, yy)
                diag_blk = Kab
                if a == b and q > 1:
                    for p in range(q):
                        if p != m and Pi[(m, p)] is not None:
                            D = tt.matmat(Pi[(m, p)], tt.transpose_mpo(Pi[(m, p)]))
                            diag_blk = tt.round_tt(tt.add(diag_blk, tt.scale(D, gamma)), eps * 1e-2)
                K = acc_add(K, attach_matrix(diag_blk, (m, m), (a, b)))
                for p in range(q):
                    if m == p or Pi[(m, p)] is None:
                        continue
                    off = tt.matmat(Pi[(m, p)], Kab)
                    if a == b:
                        off = tt.add(off, tt.scale(Pi[(m, p)], -gamma))
                    K = acc_add(K, attach_matrix(tt.round_tt(off, eps * 1e-2), (m, p), (a, b)))
    for a in (0, 1):
        for m in range(q):
            g = loads[m][a]
            for p in range(q):
                if m != p and Pi[(m, p)] is not None:
                    g = tt.add(g, tt.matvec(Pi[(m, p)], loads[p][a]))
            f = acc_add(f, attach_vector(tt.round_tt(g, eps * 1e-2), m, a))
    K = tt.round_tt(K, eps)
    f = tt.round_tt(f, eps)
    # Dirichlet masks: K <- M K M + (I - M), f <- M f
    mvec = mask_qtt(prob)
    Md = tt.diag_mpo(mvec)
    ones = [np.ones((1, G.shape[1], 1)) for G in mvec]
    IminusM = tt.diag_mpo(tt.add(ones, tt.scale(mvec, -1.0)))
    K = tt.round_tt(tt.matmat(tt.matmat(Md, K), Md), eps)
    K = tt.round_tt(tt.add(K, IminusM), eps)
    f = tt.round_tt(tt.matvec(Md, f), eps)
    return K, f
