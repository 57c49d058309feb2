"""Node numberings of Section 3.2 (oracle; test infrastructure only).

Canonical order  L_ij = i + 2^d j.
Z-order          Z_ij = [i_1, j_1, i_2, j_2, ..., i_d, j_d]_2, i_1 the least
                 significant bit (bit interleaving, Morton order).
Vector DOF maps  N_ij = (2 L_ij + 1, 2 L_ij + 2) and P_ij = (2 Z_ij + 1,
                 2 Z_ij + 2) in the paper's 1-based form.
"""
from __future__ import annotations

import numpy as np


def canonical(i, j, d: int):
    """L_ij = i + 2^d j (Section 3.2)."""
    return np.asarray(i, dtype=np.int64) + (np.int64(1) << d) * np.asarray(j, dtype=np.int64)


def zorder(i, j, d: int):
    """Z_ij = sum_k 2^(2k-2) i_k + 2^(2k-1) j_k with i = sum_k 2^(k-1) i_k
    (Section 3.2); one bit pair per level, x bit below y bit."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    z = np.zeros(np.broadcast(i, j).shape, dtype=np.int64)
    for k in range(1, d + 1):
        ik = (i >> (k - 1)) & 1
        jk = (j >> (k - 1)) & 1
        z = z + (ik << (2 * k - 2)) + (jk << (2 * k - 1))
    return z


def dof_N(i, j, d: int):
    """Canonical vector DOF pair N_ij, 1-based as printed in Section 3.2."""
    l = canonical(i, j, d)
    return 2 * l + 1, 2 * l + 2


def dof_P(i, j, d: int):
    """Z-ordered vector DOF pair P_ij, 1-based as printed in Section 3.2."""
    z = zorder(i, j, d)
    return 2 * z + 1, 2 * z + 2


def qtt_dof(i, j, m, c, d: int, q: int):
    """0-based position of DOF (node (i, j) of patch m, component c) in the
    QTT layout: d position cores (Z-order), a patch core of mode q, then a
    component core of mode 2 (block Kronecker assembly of Section 3.7 puts the
    component outermost)."""
    nn = np.int64(1) << (2 * d)
    return zorder(i, j, d) + nn * np.asarray(m, dtype=np.int64) + nn * q * np.asarray(c, dtype=np.int64)


def canonical_dof(i, j, m, c, d: int, q: int):
    """0-based position in the canonical layout: interleaved components
    2 L_ij + c (the 0-based form of N_ij) within patch m, patches in order."""
    nn = np.int64(1) << (2 * d)
    return 2 * canonical(i, j, d) + np.asarray(c, dtype=np.int64) + 2 * nn * np.asarray(m, dtype=np.int64)
