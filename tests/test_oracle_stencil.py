"""Pins of the matrix-free residual (oracle/stencil.py) against the sparse
assembly of the oracle FEM: the element-by-element product equals the
assembled patch stiffness times u, it has the three rigid-body modes in its
kernel, and the masked residual of the sparse direct solution vanishes."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, stencil


@pytest.mark.parametrize("L,E,nu", [(3, 1.0, 0.3), (5, 210.0, 0.25)])
def test_matrix_free_apply_equals_sparse_product(L, E, nu):
    n = 1 << L
    u = np.random.default_rng(L).standard_normal(2 * n * n)
    K = fem.patch_stiffness(L, E, nu)
    np.testing.assert_allclose(stencil.patch_apply(L, E, nu, u), K @ u, rtol=0, atol=1e-12 * abs(K @ u).max())


def test_matrix_free_rigid_modes():
    L = 4
    n = 1 << L
    h = 1.0 / (n - 1)
    x = np.tile(h * np.arange(n), n)              # node i + n j
    y = np.repeat(h * np.arange(n), n)
    for ux, uy in ((np.ones_like(x), 0 * x), (0 * x, np.ones_like(x)), (-y, x)):
        u = np.empty(2 * n * n)
        u[0::2], u[1::2] = ux, uy
        assert abs(stencil.patch_apply(L, 3.0, 0.3, u)).max() <= 1e-12


def test_masked_residual_of_direct_solution_vanishes():
    prob = W.plate_top_traction(6, 17.0, 0.33, 1.3, 2.0)
    K, f, free, node_map = fem.merged_system(prob)
    um = fem.solve_eliminated(K, f, free)
    n = prob.n
    g = node_map[0].ravel(order="F")               # local node i + n j -> merged node
    u = np.empty(2 * n * n)
    u[0::2], u[1::2] = um[2 * g], um[2 * g + 1]
    r, fbc = stencil.masked_residual(prob, u)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(fbc)
    # a perturbation of one free value shows up in the residual
    u[2 * (n // 2 + n * (n // 2))] += 1e-6
    r2, _ = stencil.masked_residual(prob, u)
    assert np.linalg.norm(r2) > 1e3 * np.linalg.norm(r)
