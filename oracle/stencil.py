"""O-3: matrix-free Q1 plane-stress residual on one unit-square patch
(oracle; test infrastructure only).

For patch meshes too large for sparse assembly (L = 12: 33.5 M DOFs), the
product K u is applied element by element without forming K: all (n-1)^2
elements of a patch are translates of one square element, so

    (K u)_a = sum over elements e containing node a of
              sum_b Ke[a_loc(e), b_loc(e)] u_b,

with Ke the 8x8 element stiffness of Section 3.4 (2x2 Gauss, plane stress),
is sixteen shifted 2x2 block products over the node grid.  Homogeneous
Dirichlet conditions follow the masked form of Section 3.8:
K_bc = M K M + (I - M), f_bc = M (f - K g) + g, M = diag(free), with
g = (I - M) u0 the prescribed values (zero for homogeneous conditions).  The load is the
oracle's own patch load (consistent mass x intensity, edge tractions).
Everything is plain NumPy in FP64.
"""
from __future__ import annotations

import numpy as np

from . import fem

# vertex (i, j) offsets of the element corners in the reference order of
# Section 3.4: (i, j), (i+1, j), (i+1, j+1), (i, j+1)
_OFF = ((0, 0), (1, 0), (1, 1), (0, 1))


def patch_apply(L: int, E: float, nu: float, u: np.ndarray) -> np.ndarray:
    """K^(m) u for one unit-square patch; u and the result in the local DOF
    order 2 (i + n j) + c."""
    n = 1 << L
    h = 1.0 / (n - 1)
    xy = np.array([[0.0, 0.0], [h, 0.0], [h, h], [0.0, h]])
    Ke = fem.element_stiffness(xy, fem.plane_stress_C(E, nu))
    U = u.reshape(n, n, 2)                      # [j, i, c]
    out = np.zeros_like(U)
    for a, (ia, ja) in enumerate(_OFF):
        dst = out[ja:ja + n - 1, ia:ia + n - 1]
        for b, (ib, jb) in enumerate(_OFF):
            src = U[jb:jb + n - 1, ib:ib + n - 1]
            dst += src @ Ke[2 * a:2 * a + 2, 2 * b:2 * b + 2].T
    return out.reshape(-1)


def masked_residual(prob, u: np.ndarray):
    """f_bc - K_bc u of a one-patch problem in the local DOF order; returns
    (residual, f_bc)."""
    assert prob.q == 1, "matrix-free residual covers one-patch problems"
    n = prob.n
    flags = fem.constrained_flags(prob)[0]      # [i, j]
    free = np.empty((n, n, 2), dtype=bool)      # [j, i, c]
    free[:, :, 0] = (flags.T & 1) == 0
    free[:, :, 1] = (flags.T & 2) == 0
    free = free.reshape(-1)
    f = fem.patch_load(prob, 0)
    g = np.where(free, 0.0, fem.patch_dirichlet(prob, 0))      # prescribed values, lifted
    fbc = np.where(free, f - patch_apply(prob.L, prob.E, prob.nu, g), 0.0) + g
    Ku = patch_apply(prob.L, prob.E, prob.nu, np.where(free, u, 0.0))
    r = fbc - np.where(free, Ku, 0.0) - np.where(free, 0.0, u)
    return r, fbc
