"""Pins of the O-2 tensor-train layer and the index maps: brute force on tiny
inputs, textbook QTT ranks of elementary functions, the rounding error bound
of Oseledets (2011), and the recursive (quadrant) definition of Morton
order."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import indexing, tt


# ---------------------------------------------------------------- index maps

def _morton_recursive(i, j, d):
    """Quadrant recursion: the four 2^(d-1) sub-squares are visited in the
    order (low x, low y), (high x, low y), (low x, high y), (high x, high y),
    i.e. the most significant bit pair selects the quadrant."""
    if d == 0:
        return 0
    half = 1 << (d - 1)
    quad = (i >= half) + 2 * (j >= half)
    return quad * half * half + _morton_recursive(i % half, j % half, d - 1)


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_zorder_matches_quadrant_recursion_and_is_bijective(d):
    n = 1 << d
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    z = indexing.zorder(ii, jj, d)
    ref = np.vectorize(lambda a, b: _morton_recursive(int(a), int(b), d))(ii, jj)
    np.testing.assert_array_equal(z, ref)
    assert sorted(z.ravel().tolist()) == list(range(n * n))


def test_zorder_small_example_and_dof_maps():
    # d = 1: (0,0) (1,0) (0,1) (1,1) -> 0 1 2 3; canonical i + 2 j coincides
    assert [int(indexing.zorder(i, j, 1)) for i, j in [(0, 0), (1, 0), (0, 1), (1, 1)]] == [0, 1, 2, 3]
    # d = 2: node (2, 1) has i = [0,1], j = [1,0] -> bits i1 j1 i2 j2 = 0 1 1 0 -> 6
    assert int(indexing.zorder(2, 1, 2)) == 6
    assert int(indexing.canonical(2, 1, 2)) == 6
    assert int(indexing.zorder(1, 2, 2)) == 9 and int(indexing.canonical(1, 2, 2)) == 9
    assert int(indexing.zorder(3, 0, 2)) == 5 and int(indexing.canonical(3, 0, 2)) == 3
    px, py = indexing.dof_P(3, 0, 2)
    nx, ny = indexing.dof_N(3, 0, 2)
    assert (int(px), int(py)) == (11, 12) and (int(nx), int(ny)) == (7, 8)


# ---------------------------------------------------------------- TT basics

def test_full_brute_force():
    cores = W.random_tt(3, [2, 3, 2], [1, 2, 2, 1])
    v = tt.full(cores)
    for i1 in range(2):
        for i2 in range(3):
            for i3 in range(2):
                ref = (cores[0][:, i1, :] @ cores[1][:, i2, :] @ cores[2][:, i3, :])[0, 0]
                assert v[i1 + 2 * i2 + 6 * i3] == pytest.approx(ref, abs=1e-15)


def test_full_matrix_brute_force():
    A = W.random_mpo(4, [2, 2], [3, 2], [1, 2, 1])
    M = tt.full_matrix(A)
    for i1 in range(2):
        for i2 in range(2):
            for j1 in range(3):
                for j2 in range(2):
                    ref = (A[0][:, i1, j1, :] @ A[1][:, i2, j2, :])[0, 0]
                    assert M[i1 + 2 * i2, j1 + 3 * j2] == pytest.approx(ref, abs=1e-15)


def test_tt_svd_exact_recovery_and_bound():
    modes = [4, 4, 4, 2]
    x = W.random_tt(1, modes, [1, 3, 5, 2, 1])
    v = tt.full(x)
    y = tt.tt_svd(v, modes, 1e-13)
    assert tt.ranks(y) == [1, 3, 5, 2, 1]
    np.testing.assert_allclose(tt.full(y), v, atol=1e-13 * np.abs(v).max())
    rng = np.random.default_rng(0)
    w = rng.standard_normal(4 ** 4 * 2)
    for eps in (1e-1, 1e-2, 1e-3):
        c = tt.tt_svd(w, [4, 4, 4, 4, 2], eps)
        assert np.linalg.norm(tt.full(c) - w) <= eps * np.linalg.norm(w) * (1 + 1e-12)


@pytest.mark.parametrize("L", [6, 10])
def test_qtt_ranks_of_elementary_functions(L):
    """Textbook QTT facts: exp and sin have rank 1 and 2; a degree-p
    polynomial has rank p + 1."""
    t = np.linspace(0.0, 1.0, 1 << L)
    assert tt.max_rank(tt.tt_svd(np.exp(0.7 * t), [2] * L, 1e-13)) == 1
    assert tt.max_rank(tt.tt_svd(np.sin(3.0 * t + 0.2), [2] * L, 1e-13)) == 2
    assert tt.max_rank(tt.tt_svd(1 + t - 2 * t ** 3, [2] * L, 1e-12)) == 4


def test_matvec_matmat_vs_dense():
    modes = [4, 4, 2]
    A = W.random_mpo(2, modes, modes, [1, 3, 2, 1])
    B = W.random_mpo(5, modes, modes, [1, 2, 2, 1])
    x = W.random_tt(3, modes, [1, 2, 3, 1])
    Ad, Bd = tt.full_matrix(A), tt.full_matrix(B)
    np.testing.assert_allclose(tt.full(tt.matvec(A, x)), Ad @ tt.full(x), atol=1e-14)
    np.testing.assert_allclose(tt.full_matrix(tt.matmat(A, B)), Ad @ Bd, atol=1e-14)
    np.testing.assert_allclose(tt.full_matrix(tt.transpose_mpo(A)), Ad.T, atol=0)
    d = tt.diag_mpo(x)
    np.testing.assert_allclose(tt.full_matrix(d), np.diag(tt.full(x)), atol=0)


def test_zkron_is_permuted_kron():
    """(A zkron B) = P_Z (B kron A) P_Z^T with P_Z the Morton permutation of a
    canonical (x fastest) node index."""
    L = 3
    n = 1 << L
    A = W.random_mpo(7, [2] * L, [2] * L, [1, 2, 3, 1])
    B = W.random_mpo(8, [2] * L, [2] * L, [1, 3, 2, 1])
    Z = tt.full_matrix(tt.zkron(A, B))
    canon = np.kron(tt.full_matrix(B), tt.full_matrix(A))   # index i + n j
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    lin = indexing.canonical(ii, jj, L).ravel()
    zz = indexing.zorder(ii, jj, L).ravel()
    P = np.zeros((n * n, n * n))
    P[zz, lin] = 1.0
    np.testing.assert_allclose(Z, P @ canon @ P.T, atol=1e-15)
    a = W.random_tt(9, [2] * L, [1, 2, 2, 1])
    b = W.random_tt(10, [2] * L, [1, 1, 2, 1])
    zv = tt.full(tt.zkron_vec(a, b))
    np.testing.assert_allclose(zv, P @ np.kron(tt.full(b), tt.full(a)), atol=1e-15)


def test_add_scale_kron_dot_norm():
    modes = [4, 4, 2]
    x = W.random_tt(1, modes, [1, 2, 3, 1])
    y = W.random_tt(2, modes, [1, 3, 2, 1])
    xv, yv = tt.full(x), tt.full(y)
    np.testing.assert_allclose(tt.full(tt.add(x, tt.scale(y, -2.5))), xv - 2.5 * yv, atol=1e-14)
    assert tt.dot(x, y) == pytest.approx(xv @ yv, rel=1e-12)
    assert tt.norm(x) == pytest.approx(np.linalg.norm(xv), rel=1e-13)
    k = tt.kron(x, y)
    np.testing.assert_allclose(tt.full(k), np.kron(yv, xv), atol=1e-15)


def test_norm_of_small_difference_is_accurate():
    """||x - (x + tiny y)|| via orthogonalisation keeps absolute accuracy of
    order eps ||x|| (the property the FP64 residual relies on)."""
    modes = [4, 4, 4, 2]
    x = W.random_tt(1, modes, [1, 4, 6, 2, 1])
    y = W.random_tt(2, modes, [1, 3, 3, 2, 1])
    d = tt.add(x, tt.scale(tt.add(x, tt.scale(y, 1e-9)), -1.0))
    ref = 1e-9 * np.linalg.norm(tt.full(y))
    assert tt.norm(d) == pytest.approx(ref, rel=1e-5)


def test_round_bound_and_rank_recovery():
    modes = [4, 4, 4, 4, 2]
    x = W.random_tt(11, modes, [1, 3, 6, 5, 2, 1])
    xx = tt.add(x, x)
    r = tt.round_tt(xx, 1e-12)
    assert tt.ranks(r) == tt.ranks(x)
    np.testing.assert_allclose(tt.full(r), 2 * tt.full(x), atol=1e-13)
    # padded exact low-rank tensor is recovered exactly
    pad = [np.pad(G, ((0, 2 if k else 0), (0, 0), (0, 2 if k < len(x) - 1 else 0))) for k, G in enumerate(x)]
    np.testing.assert_allclose(tt.full(pad), tt.full(x), atol=0)
    assert tt.ranks(tt.round_tt(pad, 1e-13)) == tt.ranks(x)
    rng = np.random.default_rng(1)
    w = tt.tt_svd(rng.standard_normal(4 ** 4 * 2), modes, 1e-15)
    for eps in (0.3, 0.1, 1e-2):
        c = tt.round_tt(w, eps)
        err = np.linalg.norm(tt.full(c) - tt.full(w))
        assert err <= eps * np.linalg.norm(tt.full(w)) * (1 + 1e-10)


def test_round_mpo():
    A = W.random_mpo(3, [4, 4, 2], [4, 4, 2], [1, 3, 2, 1])
    A2 = tt.add(A, A)
    r = tt.round_tt(A2, 1e-13)
    assert tt.ranks(r) == tt.ranks(A)
    np.testing.assert_allclose(tt.full_matrix(r), 2 * tt.full_matrix(A), atol=1e-13)


def test_erank_and_parameter_counts():
    """r_e solves r_e n_1 + sum r_e^2 n_i + r_e n_d = storage (Section 4):
    uniform ranks give r_e = r exactly.  N_d counts stored core entries
    (Eq. Nd); a full-rank QTT of a 2 * 4^2 = 32-entry vector (modes 4, 4, 2,
    ranks 1, 4, 2, 1) stores 16 + 32 + 4 = 52 entries, the value the paper
    prints for d = 2 in its N_d-versus-d plots (Section 5.3)."""
    x = W.random_tt(1, [4, 4, 4, 2], [1, 5, 5, 5, 1])
    assert tt.erank(x) == pytest.approx(5.0)
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_Nd_d2.txt")
    rows = [ln.split() for ln in open(golden) if ln.strip() and not ln.startswith("#")]
    d, nd, modes, ranks = rows[0]
    modes = [int(v) for v in modes.split(",")]
    ranks = [int(v) for v in ranks.split(",")]
    assert int(d) == 2 and len(modes) == int(d) + 1
    y = W.random_tt(2, modes, ranks)
    assert tt.n_params(y) == int(nd)
    assert tt.max_rank(y) == 4
