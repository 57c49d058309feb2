"""Pins of the O-2 QTT assembly (Algorithm 1) against the O-1 sparse FEM, and
of the O-2 AMEn solver against dense direct solves."""
import numpy as np
import pytest

import workloads as W
from oracle import amen, assembly, fem, tt


@pytest.mark.parametrize("make,L", [(W.plate_body_force, 3), (W.plate_traction_smooth, 4),
                                    (W.lshape_shear, 3), (W.two_patch_strip, 3)])
def test_qtt_assembly_equals_sparse_fem(make, L):
    """qtt_to_full(K) equals the assembled FE matrix to 1e-12 (relative to
    max |K|); the load vector likewise."""
    prob = make(L)
    K, f = assembly.assemble(prob)
    Kd, fd, _ = fem.duplicated_system(prob)
    Kf = tt.full_matrix(K)
    assert np.abs(Kf - Kd.toarray()).max() <= 1e-12 * np.abs(Kd).max()
    assert np.abs(tt.full(f) - fd).max() <= 1e-12 * np.abs(fd).max()


def test_patch_blocks_rigid_modes_in_qtt():
    """K^(m) (before masks) annihilates the three rigid-body modes; the modes
    are QTT vectors of rank <= 2 built from 1D grid functions, so the check
    runs in QTT at a level where dense storage is still cheap to compare."""
    L = 6
    n = 1 << L
    h = 1.0 / (n - 1)
    blocks = assembly.patch_blocks(L, 7.0, 0.3)
    one = assembly.qtt_vector_1d(np.ones(n), L)
    lin = assembly.qtt_vector_1d(h * np.arange(n), L)
    zero = tt.scale(tt.zkron_vec(one, one), 0.0)
    modes = [(tt.zkron_vec(one, one), zero), (zero, tt.zkron_vec(one, one)),
             (tt.scale(tt.zkron_vec(one, lin), -1.0), tt.zkron_vec(lin, one))]
    scale = max(np.abs(tt.full_matrix(b)).max() for b in blocks)
    for ux, uy in modes:
        rx = tt.full(tt.matvec(blocks[0], ux)) + tt.full(tt.matvec(blocks[1], uy))
        ry = tt.full(tt.matvec(blocks[2], ux)) + tt.full(tt.matvec(blocks[3], uy))
        assert max(np.abs(rx).max(), np.abs(ry).max()) <= 1e-11 * scale


def test_stiffness_ranks_do_not_grow_with_level():
    """The Z-ordered stiffness has QTT ranks bounded in the level (the rank
    advantage of Z-order, Section 3.2 and Section 5.2)."""
    r5 = tt.ranks(assembly.patch_blocks(5, 1.0, 0.3)[0])
    r8 = tt.ranks(assembly.patch_blocks(8, 1.0, 0.3)[0])
    assert max(r8) == max(r5)


@pytest.mark.parametrize("make,L", [(W.plate_body_force, 3), (W.lshape_shear, 2)])
def test_amen_equals_direct_solve(make, L):
    prob = make(L)
    K, f = assembly.assemble(prob)
    Kd = tt.full_matrix(K)
    fd = tt.full(f)
    u = np.linalg.solve(Kd, fd)
    modes = W.qtt_modes(prob)
    x0 = W.random_tt(5, modes, [1] + [2] * (len(modes) - 1) + [1])
    z0 = W.random_tt(6, modes, [1] + [4] * (len(modes) - 1) + [1])
    eps = 1e-10
    x, info = amen.amen_solve(K, f, x0, z0, eps, max_sweeps=20)
    assert info.converged
    xf = tt.full(x)
    res = np.linalg.norm(Kd @ xf - fd) / np.linalg.norm(fd)
    kappa = np.linalg.cond(Kd)
    assert res <= 10 * eps * np.sqrt(len(modes))
    assert np.linalg.norm(xf - u) / np.linalg.norm(u) <= kappa * res * 1.01


def test_amen_local_helpers_match_dense():
    """The local operator applied by contraction equals the explicit dense
    local matrix, and both equal the Galerkin projection P^T K P of the full
    matrix onto the frame of the current core."""
    prob = W.plate_body_force(2)
    K, f = assembly.assemble(prob)
    modes = W.qtt_modes(prob)
    x = tt.right_orthogonalize(W.random_tt(2, modes, [1, 3, 4, 1]), 0)
    x = tt.left_orthogonalize(x, 1)               # core 1 is the free core
    k = 1
    PhiL = amen._left_XAX(np.ones((1, 1, 1)), x[0], K[0], x[0])
    PhiR = amen._right_XAX(np.ones((1, 1, 1)), x[2], K[2], x[2])
    B = amen.local_matrix(PhiL, K[1], PhiR)
    # frame P = X_<k kron I kron X_>k as a dense matrix: rows (i, j, k) with
    # the first core's index fastest, columns (a, c, b) with a fastest
    left = x[0][0]                                 # (4, r1)
    right = x[2][:, :, 0]                          # (r2, 2)
    n = 4
    r1, r2 = left.shape[1], right.shape[0]
    P = np.einsum("ia,jc,bk->kjibca", left, np.eye(n), right).reshape(4 * n * 2, r1 * n * r2)
    Kd = tt.full_matrix(K)
    np.testing.assert_allclose(B, P.T @ Kd @ P, atol=1e-10 * np.abs(Kd).max())
    v = np.random.default_rng(0).standard_normal((r1, n, r2))
    np.testing.assert_allclose(amen.local_apply(PhiL, K[1], PhiR, v).reshape(-1, order="F"),
                               B @ v.reshape(-1, order="F"), atol=1e-10 * np.abs(Kd).max())


@pytest.mark.parametrize("make,L", [(W.plate_body_force, 7), (W.lshape_shear, 6)])
def test_transpose_identity_at_large_level(make, L):
    """<K x, y> = <x, K^T y> in QTT arithmetic at levels too large for dense
    checks (a transposed operand or swapped mode pair in the matvec or the
    MPO transpose breaks it for the non-symmetric multi-patch K); for one
    patch K is symmetric, so <K x, y> = <x, K y> as well."""
    prob = make(L)
    K, _ = assembly.assemble(prob)
    modes = W.qtt_modes(prob)
    x = W.random_tt(31, modes, [1] + [3] * (len(modes) - 1) + [1])
    y = W.random_tt(32, modes, [1] + [4] * (len(modes) - 1) + [1])
    lhs = tt.dot(tt.matvec(K, x), y)
    rhs = tt.dot(x, tt.matvec(tt.transpose_mpo(K), y))
    scale = tt.norm(tt.matvec(K, x)) * tt.norm(y)
    assert abs(lhs - rhs) <= 1e-12 * scale
    if prob.q == 1:
        assert abs(lhs - tt.dot(x, tt.matvec(K, y))) <= 1e-12 * scale
    else:
        # the concatenated system is not symmetric: the identity is not trivial
        assert abs(lhs - tt.dot(x, tt.matvec(K, y))) > 1e-8 * scale
