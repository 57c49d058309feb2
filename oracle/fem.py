"""O-1: sparse Q1 plane-stress finite elements (oracle; test infrastructure).

Follows Section 3 of the paper:
  * element stiffness  K_c1c2 = int B_c1^T C B_c2 |J| over the reference
    square, 2x2 tensor Gauss rule (Sections 3.3.2 and 3.4, Eq. Kc1c2:def);
  * plane-stress constitutive matrix C (Eq. Cmat; entries are the textbook
    plane-stress values, which the paper leaves implicit);
  * load = consistent mass x nodal intensity (Eq. load:vector:intensity),
    plus edge traction int t.v ds (weak form, Eq. weak:general) by the 1D
    consistent edge mass;
  * Dirichlet conditions by elimination (Section 3.8 masks are the
    QTT-side equivalent);
  * multi-patch systems assembled two ways:
      merged      -- coincident nodes merged (conforming FEM, SPD);
      duplicated  -- the paper's concatenation (Sections 3.3.1 and 3.6):
                     every copy of a shared node carries the summed
                     equilibrium row plus gamma (D u_copy - sum partners).
Everything is plain SciPy sparse assembly and a sparse direct solve.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import indexing

# Reference corners in the counter-clockwise order of Section 3.4:
# (-1,-1) -> vertex 1, (1,-1) -> 2, (1,1) -> 3, (-1,1) -> 4.
_CORNERS = np.array([(-1.0, -1.0), (1.0, -1.0), (1.0, 1.0), (-1.0, 1.0)])
_G = 1.0 / math.sqrt(3.0)
_GAUSS2 = [(-_G, 1.0), (_G, 1.0)]


def plane_stress_C(E: float, nu: float) -> np.ndarray:
    """Voigt constitutive matrix of Eq. Cmat for plane stress."""
    e = E / (1.0 - nu * nu)
    return e * np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, 0.5 * (1.0 - nu)]])


def lame(E: float, nu: float) -> Tuple[float, float]:
    """Lame constants lambda, mu of Section 2."""
    return E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def shape(xi: float, eta: float) -> np.ndarray:
    """Bilinear shape functions Phi_c at (xi, eta), corner order of _CORNERS."""
    return np.array([(1 + cx * xi) * (1 + cy * eta) / 4.0 for cx, cy in _CORNERS])


def shape_grad(xi: float, eta: float) -> np.ndarray:
    """(dPhi/dxi, dPhi/deta) for the four corners, shape (2, 4)."""
    return np.array([[cx * (1 + cy * eta) / 4.0 for cx, cy in _CORNERS],
                     [cy * (1 + cx * xi) / 4.0 for cx, cy in _CORNERS]])


def element_stiffness(xy: np.ndarray, C: np.ndarray) -> np.ndarray:
    """8x8 element matrix, DOFs (ux1, uy1, ..., ux4, uy4).

    xy : (4, 2) vertex coordinates in reference-corner order.
    Quadrature of B^T C B |J| with the 2x2 Gauss rule (Section 3.4)."""
    Ke = np.zeros((8, 8))
    for xi, wx in _GAUSS2:
        for eta, wy in _GAUSS2:
            dN = shape_grad(xi, eta)            # (2, 4) d/dxi, d/deta
            J = dN @ xy                         # [[dx/dxi, dy/dxi], [dx/deta, dy/deta]]
            detJ = np.linalg.det(J)
            dNxy = np.linalg.solve(J, dN)       # rows d/dx, d/dy
            B = np.zeros((3, 8))
            B[0, 0::2] = dNxy[0]
            B[1, 1::2] = dNxy[1]
            B[2, 0::2] = dNxy[1]
            B[2, 1::2] = dNxy[0]
            Ke += wx * wy * (B.T @ C @ B) * detJ
    return Ke


def element_mass(xy: np.ndarray) -> np.ndarray:
    """4x4 scalar element mass int Phi_c1 Phi_c2 |J| (2x2 Gauss), the matrix
    G_c1c2 of Section 3.5."""
    Me = np.zeros((4, 4))
    for xi, wx in _GAUSS2:
        for eta, wy in _GAUSS2:
            N = shape(xi, eta)
            J = shape_grad(xi, eta) @ xy
            Me += wx * wy * np.outer(N, N) * np.linalg.det(J)
    return Me


def edge_mass(length: float) -> np.ndarray:
    """2x2 consistent mass of a straight edge segment (2-point Gauss)."""
    Me = np.zeros((2, 2))
    for s, w in _GAUSS2:
        N = np.array([(1 - s) / 2.0, (1 + s) / 2.0])
        Me += w * np.outer(N, N) * (length / 2.0)
    return Me


def _body_factor(kind: int, t: np.ndarray) -> np.ndarray:
    if kind == 0:
        return np.ones_like(t)
    if kind == 1:
        return t.copy()
    if kind == 2:
        return np.sin(math.pi * t)
    if kind == 3:
        return np.cos(math.pi * t)
    if kind == 4:
        return t * t
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# Per-patch matrices in a local (i, j, c) numbering
# ----------------------------------------------------------------------------

def _patch_nodes(n: int):
    """Node (i, j) -> local id i + n j (canonical order)."""
    return np.arange(n * n).reshape(n, n).T    # [i, j] -> i + n j


def patch_stiffness(L: int, E: float, nu: float, origin=(0.0, 0.0)) -> sp.csr_matrix:
    """K^(m) of one unit-square patch with n = 2^L nodes per side, local DOF
    index 2 (i + n j) + c (Eq. eq-stiffness assembled over elements)."""
    n = 1 << L
    h = 1.0 / (n - 1)
    C = plane_stress_C(E, nu)
    nid = _patch_nodes(n)
    ii, jj = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    # vertex node ids in reference-corner order
    verts = np.stack([nid[ii, jj], nid[ii + 1, jj], nid[ii + 1, jj + 1], nid[ii, jj + 1]], axis=1)
    # all elements of a patch are translates of each other: one element matrix
    x0, y0 = origin
    xy = np.array([[x0, y0], [x0 + h, y0], [x0 + h, y0 + h], [x0, y0 + h]])
    Ke = element_stiffness(xy, C)
    dofs = np.empty((verts.shape[0], 8), dtype=np.int64)
    dofs[:, 0::2] = 2 * verts
    dofs[:, 1::2] = 2 * verts + 1
    rows = np.repeat(dofs, 8, axis=1).ravel()
    cols = np.tile(dofs, (1, 8)).ravel()
    vals = np.tile(Ke.ravel(), verts.shape[0])
    N = 2 * n * n
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def patch_mass(L: int) -> sp.csr_matrix:
    """Scalar consistent mass of one patch, local node index i + n j."""
    n = 1 << L
    h = 1.0 / (n - 1)
    nid = _patch_nodes(n)
    ii, jj = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    verts = np.stack([nid[ii, jj], nid[ii + 1, jj], nid[ii + 1, jj + 1], nid[ii, jj + 1]], axis=1)
    xy = np.array([[0, 0], [h, 0], [h, h], [0, h]], dtype=float)
    Me = element_mass(xy)
    rows = np.repeat(verts, 4, axis=1).ravel()
    cols = np.tile(verts, (1, 4)).ravel()
    vals = np.tile(Me.ravel(), verts.shape[0])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n * n, n * n))


def _side_nodes(n: int, side: int):
    """(i, j) arrays of the nodes on a patch side, ordered along the side."""
    t = np.arange(n)
    if side == 0:
        return np.zeros(n, dtype=np.int64), t
    if side == 1:
        return np.full(n, n - 1, dtype=np.int64), t
    if side == 2:
        return t, np.zeros(n, dtype=np.int64)
    if side == 3:
        return t, np.full(n, n - 1, dtype=np.int64)
    raise ValueError(side)


def patch_load(prob, m: int) -> np.ndarray:
    """f^(m) in local DOF order 2 (i + n j) + c: consistent mass x nodal body
    force intensity (Eq. load:vector:intensity) plus edge tractions."""
    L = prob.L
    n = 1 << L
    h = 1.0 / (n - 1)
    ox, oy = prob.patches[m]
    x = ox + h * np.arange(n)
    y = oy + h * np.arange(n)
    f = np.zeros(2 * n * n)
    if prob.body:
        M = patch_mass(L)
        for comp, coeff, kx, ky in prob.body:
            fbar = coeff * np.outer(_body_factor(kx, x), _body_factor(ky, y))  # [i, j]
            fbar_vec = fbar.T.ravel()                                        # i + n j
            f[comp::2] += M @ fbar_vec
    Me = edge_mass(h)
    for (pm, side, tx, ty) in prob.traction:
        if pm != m:
            continue
        ii, jj = _side_nodes(n, side)
        w = np.zeros(n)
        for e in range(n - 1):
            w[e:e + 2] += Me @ np.ones(2)
        nodes = ii + n * jj
        f[2 * nodes] += w * tx
        f[2 * nodes + 1] += w * ty
    return f


def patch_dirichlet(prob, m: int) -> np.ndarray:
    """Nodal values of the prescribed displacement u0 (Algorithm 1 input) on
    patch m in local DOF order 2 (i + n j) + c; only constrained DOFs use
    them."""
    n = prob.n
    h = 1.0 / (n - 1)
    ox, oy = prob.patches[m]
    x = ox + h * np.arange(n)
    y = oy + h * np.arange(n)
    u = np.zeros(2 * n * n)
    for comp, coeff, kx, ky in prob.dirichlet:
        v = coeff * np.outer(_body_factor(kx, x), _body_factor(ky, y))   # [i, j]
        u[comp::2] += v.T.ravel()
    return u


# ----------------------------------------------------------------------------
# Constraints and coincidence
# ----------------------------------------------------------------------------

def _global_grid(prob, m: int):
    """Integer global grid coordinates (I, J) of patch m's nodes, [i, j]."""
    n = prob.n
    ox, oy = prob.patches[m]
    I = ox * (n - 1) + np.arange(n)
    J = oy * (n - 1) + np.arange(n)
    return np.meshgrid(I, J, indexing="ij")


def constrained_flags(prob) -> List[np.ndarray]:
    """Per patch, an (n, n) int array of FIX flags at each node: the union of
    the flags of every side (of every patch) through that physical point, so
    that all copies of a shared node carry the same constraint."""
    n = prob.n
    own = []
    for m in range(prob.q):
        fl = np.zeros((n, n), dtype=np.int64)
        for side, flag in enumerate(prob.bc[m]):
            if flag:
                ii, jj = _side_nodes(n, side)
                fl[ii, jj] |= flag
        own.append(fl)
    glob: Dict[Tuple[int, int], int] = {}
    for m in range(prob.q):
        I, J = _global_grid(prob, m)
        nz = np.nonzero(own[m])
        for a, b in zip(*nz):
            key = (int(I[a, b]), int(J[a, b]))
            glob[key] = glob.get(key, 0) | int(own[m][a, b])
    out = []
    for m in range(prob.q):
        I, J = _global_grid(prob, m)
        fl = own[m].copy()
        for (gi, gj), flag in glob.items():
            i = gi - prob.patches[m][0] * (n - 1)
            j = gj - prob.patches[m][1] * (n - 1)
            if 0 <= i < n and 0 <= j < n:
                fl[i, j] |= flag
        out.append(fl)
    return out


def coincidences(prob) -> List[Tuple[int, int, int, int]]:
    """All ordered pairs of distinct copies of one physical node:
    (m, local node a of m, p, local node b of p) with a, b = i + n j."""
    n = prob.n
    where: Dict[Tuple[int, int], List[Tuple[int, int]]] = {}
    for m in range(prob.q):
        I, J = _global_grid(prob, m)
        # only patch-boundary nodes can coincide with another patch
        border = np.zeros((n, n), dtype=bool)
        border[0, :] = border[-1, :] = border[:, 0] = border[:, -1] = True
        for a, b in zip(*np.nonzero(border)):
            where.setdefault((int(I[a, b]), int(J[a, b])), []).append((m, int(a + n * b)))
    pairs = []
    for copies in where.values():
        if len(copies) < 2:
            continue
        for (m, a) in copies:
            for (p, b) in copies:
                if m != p:
                    pairs.append((m, a, p, b))
    return pairs


# ----------------------------------------------------------------------------
# Global systems
# ----------------------------------------------------------------------------

def mean_diag_Kxx(prob) -> float:
    """Mean diagonal of K^(m)_xx for one patch: the default penalty gamma of
    Section 3.6."""
    K = patch_stiffness(prob.L, prob.E, prob.nu)
    return float(K.diagonal()[0::2].mean())


def duplicated_system(prob, masked: bool = True):
    """The concatenated multi-patch system in QTT DOF order (Z-order position,
    then patch, then component).

    Row of a copy a of patch m (reading of Sections 3.3.1 and 3.6):
        sum over copies s of a's node of (K^(s) u_s)_s
        + gamma (D_a u_a - sum of partner copies u_b)    [components x, y]
      = sum over copies s of f^(s)_s.
    With masked=True the homogeneous Dirichlet masks are applied as
    K <- M K M + (I - M), f <- M f (Section 3.8).
    Returns (K csr, f, free-mask bool array)."""
    L, q, n = prob.L, prob.q, prob.n
    nn = n * n
    N = 2 * q * nn
    gamma = prob.gamma if prob.gamma != 0.0 else mean_diag_Kxx(prob)
    # local DOF 2 (i + n j) + c  ->  QTT DOF
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    loc_node = (ii + n * jj).ravel()
    perm_node = np.empty(nn, dtype=np.int64)
    perm_node[loc_node] = indexing.zorder(ii.ravel(), jj.ravel(), L)
    blocks = []
    f = np.zeros(N)
    u0 = np.zeros(N)
    for m in range(q):
        Km = patch_stiffness(L, prob.E, prob.nu).tocoo()
        node_r, c_r = Km.row // 2, Km.row % 2
        node_c, c_c = Km.col // 2, Km.col % 2
        rows = perm_node[node_r] + nn * m + nn * q * c_r
        cols = perm_node[node_c] + nn * m + nn * q * c_c
        blocks.append(sp.coo_matrix((Km.data, (rows, cols)), shape=(N, N)))
        fm = patch_load(prob, m)
        um = patch_dirichlet(prob, m)
        for c in range(2):
            f[perm_node[np.arange(nn)] + nn * m + nn * q * c] += fm[c::2]
            u0[perm_node[np.arange(nn)] + nn * m + nn * q * c] = um[c::2]
    Kblk = sp.csr_matrix((N, N))
    for b in blocks:
        Kblk = Kblk + b.tocsr()
    # S = I + Pi (sum over copies), G = D - Pi (graph Laplacian on copies)
    pr, pc = [], []
    for (m, a, p, b) in coincidences(prob):
        for c in range(2):
            pr.append(perm_node[a] + nn * m + nn * q * c)
            pc.append(perm_node[b] + nn * p + nn * q * c)
    Pi = sp.csr_matrix((np.ones(len(pr)), (pr, pc)), shape=(N, N))
    D = sp.diags(np.asarray(Pi.sum(axis=1)).ravel())
    S = sp.identity(N, format="csr") + Pi
    K = S @ Kblk + gamma * (D - Pi)
    f = S @ f
    free = np.ones(N, dtype=bool)
    flags = constrained_flags(prob)
    for m in range(q):
        fl = flags[m]
        for c, bit in ((0, 1), (1, 2)):
            idx = np.nonzero((fl & bit).ravel(order="F"))[0]   # local node i + n j
            free[perm_node[idx] + nn * m + nn * q * c] = False
    if masked:
        # lifting of the prescribed values g = (I - M) u0 (Section 3.8 masks,
        # Algorithm 1's u0): free rows get M (f - K g), constrained rows g
        g = np.where(free, 0.0, u0)
        f = (f - K @ g) * free + g
        Mk = sp.diags(free.astype(float))
        K = Mk @ K @ Mk + sp.diags((~free).astype(float))
    return sp.csr_matrix(K), f, free


def merged_system(prob):
    """Conforming FEM on merged nodes.  Returns (K, f, free, node_map) where
    node_map[m] is an (n, n) array of global node ids of patch m's nodes and
    global DOF = 2 * node + c."""
    n, q = prob.n, prob.q
    ids: Dict[Tuple[int, int], int] = {}
    node_map = []
    for m in range(q):
        I, J = _global_grid(prob, m)
        nm = np.empty((n, n), dtype=np.int64)
        for a in range(n):
            for b in range(n):
                key = (int(I[a, b]), int(J[a, b]))
                if key not in ids:
                    ids[key] = len(ids)
                nm[a, b] = ids[key]
        node_map.append(nm)
    Nn = len(ids)
    N = 2 * Nn
    K = sp.csr_matrix((N, N))
    f = np.zeros(N)
    for m in range(q):
        Km = patch_stiffness(prob.L, prob.E, prob.nu).tocoo()
        g = node_map[m].ravel(order="F")          # local node i + n j -> global node
        rows = 2 * g[Km.row // 2] + Km.row % 2
        cols = 2 * g[Km.col // 2] + Km.col % 2
        K = K + sp.csr_matrix((Km.data, (rows, cols)), shape=(N, N))
        fm = patch_load(prob, m)
        np.add.at(f, 2 * g[np.arange(n * n)] + 0, fm[0::2])
        np.add.at(f, 2 * g[np.arange(n * n)] + 1, fm[1::2])
    free = np.ones(N, dtype=bool)
    flags = constrained_flags(prob)
    for m in range(q):
        fl = flags[m].ravel(order="F")
        g = node_map[m].ravel(order="F")
        free[2 * g[(fl & 1) != 0]] = False
        free[2 * g[(fl & 2) != 0] + 1] = False
    return K, f, free, node_map


def solve_eliminated(K, f, free, u_fixed=None):
    """Dirichlet by elimination: K_ff u_f = f_f - K_fc u_c; sparse direct."""
    N = K.shape[0]
    u = np.zeros(N) if u_fixed is None else np.array(u_fixed, dtype=float)
    fi = np.nonzero(free)[0]
    ci = np.nonzero(~free)[0]
    rhs = f[fi] - (K[fi][:, ci] @ u[ci] if len(ci) else 0.0)
    Kff = sp.csc_matrix(K[fi][:, fi])
    u[fi] = spla.spsolve(Kff, rhs, permc_spec="MMD_AT_PLUS_A")
    return u


def solve_merged(prob) -> Tuple[np.ndarray, list]:
    K, f, free, node_map = merged_system(prob)
    u_fixed = None
    if prob.dirichlet:
        u_fixed = np.zeros(K.shape[0])
        for m in range(prob.q):
            g = node_map[m].ravel(order="F")            # local node i + n j -> merged node
            um = patch_dirichlet(prob, m)
            u_fixed[2 * g] = um[0::2]
            u_fixed[2 * g + 1] = um[1::2]
        u_fixed = np.where(free, 0.0, u_fixed)
    return solve_eliminated(K, f, free, u_fixed), node_map


def merged_to_qtt(prob, u_merged: np.ndarray, node_map) -> np.ndarray:
    """Spread a merged-node solution onto every copy, QTT DOF order."""
    n, q, L = prob.n, prob.q, prob.L
    nn = n * n
    out = np.zeros(2 * q * nn)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    z = indexing.zorder(ii, jj, L)
    for m in range(q):
        for c in range(2):
            out[(z + nn * m + nn * q * c).ravel()] = u_merged[2 * node_map[m].ravel() + c]
    return out


def solve_duplicated(prob) -> np.ndarray:
    """Solution of the concatenated system (masked form), QTT DOF order."""
    K, f, free = duplicated_system(prob, masked=True)
    return spla.spsolve(sp.csc_matrix(K), f)
