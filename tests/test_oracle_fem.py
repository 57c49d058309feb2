"""Pins of the O-1 sparse FEM oracle against what the paper and textbook FE
theory fix: the textbook Q1 plane-stress element matrix, the patch test,
symmetry and the three rigid-body modes, O(h^2) convergence on a
manufactured solution, and the concatenated (duplicated-node) multi-patch
system reproducing the conforming solution for any penalty gamma."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fem


def _square(h):
    return np.array([[0, 0], [h, 0], [h, h], [0, h]], dtype=float)


def test_plane_stress_matrix_and_lame():
    E, nu = 2.5, 0.3
    C = fem.plane_stress_C(E, nu)
    # plane stress: sigma_zz = 0 gives C11 = 4 mu (lambda + mu) / (lambda + 2 mu)
    lam, mu = fem.lame(E, nu)
    assert C[0, 0] == pytest.approx(4 * mu * (lam + mu) / (lam + 2 * mu))
    assert C[2, 2] == pytest.approx(mu)
    assert C[0, 1] == pytest.approx(2 * mu * lam / (lam + 2 * mu))


@pytest.mark.parametrize("h", [1.0, 0.25, 1.0 / 31])
def test_element_stiffness_textbook_diagonal_and_modes(h):
    """Square Q1 plane-stress element: textbook diagonal E/(1-nu^2)(1/2 - nu/6),
    independent of the element size; symmetric; exactly three zero modes."""
    E, nu = 3.0, 0.27
    Ke = fem.element_stiffness(_square(h), fem.plane_stress_C(E, nu))
    e = E / (1 - nu * nu)
    np.testing.assert_allclose(np.diag(Ke), e * (0.5 - nu / 6) * np.ones(8), rtol=1e-13)
    # textbook x-x couplings of corner 1 with corners 2 (along x), 3
    # (diagonal) and 4 (along y), and its own x-y coupling
    assert Ke[0, 2] == pytest.approx(e * (-0.25 - nu / 12), rel=1e-12)
    assert Ke[0, 4] == pytest.approx(e * (-0.25 + nu / 12), rel=1e-12)
    assert Ke[0, 6] == pytest.approx(e * nu / 6, rel=1e-12)
    assert Ke[0, 1] == pytest.approx(e * (0.125 + nu / 8), rel=1e-12)
    np.testing.assert_allclose(Ke, Ke.T, atol=1e-14 * e)
    xy = _square(h)
    modes = [np.tile([1.0, 0.0], 4), np.tile([0.0, 1.0], 4),
             np.ravel(np.stack([-xy[:, 1], xy[:, 0]], axis=1))]
    for r in modes:
        np.testing.assert_allclose(Ke @ r, 0.0, atol=1e-12 * e)
    ev = np.linalg.eigvalsh(Ke)
    assert np.sum(np.abs(ev) < 1e-10 * e) == 3


def test_element_matrix_equals_tensor_product_form():
    """On a square, 2x2 Gauss is exact: Ke equals the analytic tensor-product
    integrals of 1D Q1 element matrices (stiffness [[1,-1],[-1,1]]/h, mass
    h/6 [[2,1],[1,2]], mixed int phi_a' phi_b = [[-1/2,-1/2],[1/2,1/2]])."""
    h = 0.2
    E, nu = 1.7, 0.21
    C = fem.plane_stress_C(E, nu)
    Ke = fem.element_stiffness(_square(h), C)
    S1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    M1 = h / 6 * np.array([[2.0, 1.0], [1.0, 2.0]])
    G1 = np.array([[-0.5, -0.5], [0.5, 0.5]])        # G1[a, b] = int phi_a' phi_b
    corners = [(0, 0), (1, 0), (1, 1), (0, 1)]
    ref = np.zeros((8, 8))
    for A, (ax, ay) in enumerate(corners):
        for B, (bx, by) in enumerate(corners):
            xx = C[0, 0] * S1[ax, bx] * M1[ay, by] + C[2, 2] * M1[ax, bx] * S1[ay, by]
            yy = C[1, 1] * M1[ax, bx] * S1[ay, by] + C[2, 2] * S1[ax, bx] * M1[ay, by]
            # test x (row), trial y (col): C12 d_x v d_y u + C33 d_y v d_x u
            xy = C[0, 1] * G1[ax, bx] * G1[by, ay] + C[2, 2] * G1[bx, ax] * G1[ay, by]
            yx = C[0, 1] * G1[bx, ax] * G1[ay, by] + C[2, 2] * G1[ax, bx] * G1[by, ay]
            ref[2 * A, 2 * B] = xx
            ref[2 * A + 1, 2 * B + 1] = yy
            ref[2 * A, 2 * B + 1] = xy
            ref[2 * A + 1, 2 * B] = yx
    np.testing.assert_allclose(Ke, ref, atol=1e-13 * np.abs(ref).max())


def test_element_mass_textbook():
    h = 0.5
    Me = fem.element_mass(_square(h))
    # bilinear mass on a square: h^2/36 [[4,2,1,2],...]
    ref = h * h / 36 * np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]], dtype=float)
    np.testing.assert_allclose(Me, ref, rtol=1e-13)


def test_patch_stiffness_symmetric_with_rigid_modes():
    L = 4
    K = fem.patch_stiffness(L, 5.0, 0.3)
    assert abs(K - K.T).max() < 1e-12
    n = 1 << L
    h = 1.0 / (n - 1)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = (ii * h).ravel(order="F")
    y = (jj * h).ravel(order="F")
    N = 2 * n * n
    for ux, uy in [(np.ones_like(x), 0 * x), (0 * x, np.ones_like(x)), (-y, x)]:
        u = np.zeros(N)
        u[0::2], u[1::2] = ux, uy
        assert np.abs(K @ u).max() < 1e-11 * abs(K).max()
    # exactly three zero eigenvalues (no hourglass modes with 2x2 Gauss)
    ev = np.linalg.eigvalsh(K.toarray())
    assert np.sum(np.abs(ev) < 1e-9 * ev.max()) == 3


def test_patch_test_linear_field():
    """Linear displacement imposed on the whole boundary, no load: the FE
    solution reproduces the linear field at every interior node."""
    L = 4
    prob = W.Problem(L=L, patches=[(0, 0)], E=2.0, nu=0.25,
                     bc=[(W.CLAMP, W.CLAMP, W.CLAMP, W.CLAMP)])
    K, f, free, node_map = fem.merged_system(prob)
    n = prob.n
    h = 1.0 / (n - 1)
    u_exact = np.zeros(K.shape[0])
    for i in range(n):
        for j in range(n):
            x, y = i * h, j * h
            g = node_map[0][i, j]
            u_exact[2 * g] = 0.1 + 0.3 * x - 0.2 * y
            u_exact[2 * g + 1] = -0.05 + 0.15 * x + 0.4 * y
    u = fem.solve_eliminated(K, f, free, u_fixed=np.where(free, 0.0, u_exact))
    np.testing.assert_allclose(u, u_exact, atol=1e-12)


def _manufactured(E, nu, L):
    """u = (sin(pi x) sin(pi y), x(1-x) y(1-y)), clamped on all sides, with
    f = -div sigma(u) written out for the plane-stress C."""
    C = fem.plane_stress_C(E, nu)
    c11, c12, c22, c33 = C[0, 0], C[0, 1], C[1, 1], C[2, 2]
    pi2 = math.pi ** 2
    body = [
        (0, (c11 + c33) * pi2, W.SINPI, W.SINPI),
        (0, -(c12 + c33), W.ONE, W.ONE), (0, 2 * (c12 + c33), W.LIN, W.ONE),
        (0, 2 * (c12 + c33), W.ONE, W.LIN), (0, -4 * (c12 + c33), W.LIN, W.LIN),
        (1, -(c12 + c33) * pi2, W.COSPI, W.COSPI),
        (1, 2 * c33, W.ONE, W.LIN), (1, -2 * c33, W.ONE, W.QUAD),
        (1, 2 * c22, W.LIN, W.ONE), (1, -2 * c22, W.QUAD, W.ONE),
    ]
    return W.Problem(L=L, patches=[(0, 0)], E=E, nu=nu,
                     bc=[(W.CLAMP, W.CLAMP, W.CLAMP, W.CLAMP)], body=body)


def test_h2_convergence_manufactured():
    """L2 error of the FE solution decreases like h^2 (slope 2 in log-log)."""
    E, nu = 1.0, 0.3
    errs, hs = [], []
    for L in range(3, 8):
        prob = _manufactured(E, nu, L)
        u, node_map = fem.solve_merged(prob)
        n = prob.n
        h = 1.0 / (n - 1)
        x = np.arange(n) * h
        X, Y = np.meshgrid(x, x, indexing="ij")
        ex = np.sin(math.pi * X) * np.sin(math.pi * Y)
        ey = X * (1 - X) * Y * (1 - Y)
        g = node_map[0].ravel(order="F")
        dx = u[2 * g] - ex.ravel(order="F")
        dy = u[2 * g + 1] - ey.ravel(order="F")
        M = fem.patch_mass(L)
        errs.append(math.sqrt(dx @ (M @ dx) + dy @ (M @ dy)))
        hs.append(h)
    slopes = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all(np.abs(slopes[-2:] - 2.0) < 0.15), slopes


@pytest.mark.parametrize("make", [W.lshape_shear, W.two_patch_strip])
def test_duplicated_equals_merged(make):
    prob = make(4)
    u, node_map = fem.solve_merged(prob)
    uq = fem.merged_to_qtt(prob, u, node_map)
    ud = fem.solve_duplicated(prob)
    assert np.abs(ud - uq).max() <= 1e-10 * np.abs(uq).max()


def test_duplicated_invariant_under_gamma():
    prob = W.lshape_shear(3)
    u1 = fem.solve_duplicated(prob)
    g = fem.mean_diag_Kxx(prob)
    prob.gamma = 2 * g
    u2 = fem.solve_duplicated(prob)
    prob.gamma = -0.5 * g          # any nonzero gamma enforces the copies' equality
    u3 = fem.solve_duplicated(prob)
    assert np.abs(u1 - u2).max() <= 1e-10 * np.abs(u1).max()
    assert np.abs(u1 - u3).max() <= 1e-10 * np.abs(u1).max()


def test_duplicated_is_nonsymmetric_multipatch_and_symmetric_single():
    K1, _, _ = fem.duplicated_system(W.plate_body_force(3))
    assert abs(K1 - K1.T).max() < 1e-12
    K3, _, _ = fem.duplicated_system(W.lshape_shear(3))
    assert abs(K3 - K3.T).max() > 1e-3


def test_load_total_force():
    """The consistent load distributes the total force exactly: sum of f_y for
    body force (0, -1) on the unit square is -1; a unit traction on an edge of
    unit length sums to 1."""
    prob = W.plate_body_force(4)
    f = fem.patch_load(prob, 0)
    assert f[1::2].sum() == pytest.approx(-1.0, rel=1e-13)
    prob2 = W.Problem(L=4, patches=[(0, 0)], E=1.0, nu=0.3, bc=[(W.CLAMP, 0, 0, 0)],
                      traction=[(0, W.TOP, 0.0, 1.0)])
    f2 = fem.patch_load(prob2, 0)
    assert f2[1::2].sum() == pytest.approx(1.0, rel=1e-13)
    assert abs(f2[0::2]).max() == 0.0


@pytest.mark.parametrize("patches", [((0, 0),), ((0, 0), (1, 0), (0, 1))])
def test_patch_test_through_the_masked_duplicated_system(patches):
    """Prescribed linear displacement on every outer side, no loads: the
    masked concatenated system with the lifting f_bc = M (f - K g) + g
    returns the linear field at every copy of every node (Q1 reproduces
    linear fields exactly), one patch and the L-shape."""
    import workloads as W
    from oracle import indexing
    prob = W.patch_test(3, patches)
    K, f, free = fem.duplicated_system(prob)
    u = spla.spsolve(sp.csc_matrix(K), f)
    n, q = prob.n, prob.q
    nn = n * n
    h = 1.0 / (n - 1)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    z = indexing.zorder(ii, jj, prob.L)
    for m, (ox, oy) in enumerate(prob.patches):
        x, y = ox + h * ii, oy + h * jj
        ux = u[(z + nn * m).ravel()]
        uy = u[(z + nn * m + nn * q).ravel()]
        np.testing.assert_allclose(ux, (0.1 + 0.2 * x - 0.3 * y).ravel(), atol=1e-12)
        np.testing.assert_allclose(uy, (-0.05 + 0.1 * x + 0.25 * y).ravel(), atol=1e-12)


def test_prescribed_edge_duplicated_equals_merged():
    """A nonzero prescribed edge: the masked duplicated system and Dirichlet
    by elimination on the merged system give the same displacements."""
    import workloads as W
    prob = W.plate_prescribed_edge(4)
    ud = fem.solve_duplicated(prob)
    um, nm = fem.solve_merged(prob)
    np.testing.assert_allclose(ud, fem.merged_to_qtt(prob, um, nm), rtol=0, atol=1e-12 * abs(ud).max())
    assert abs(ud).max() > 1e-3


def test_manufactured_plate_load_is_the_exact_body_force():
    """The body force of workloads.plate_manufactured is -div sigma of
    u = (sin pi x sin pi y, 0): the sparse FE solution converges to u at
    O(h^2) in the nodal max norm."""
    import workloads as W
    errs = []
    for L in (4, 5, 6):
        prob = W.plate_manufactured(L, E=3.0, nu=0.25)
        um, nm = fem.solve_merged(prob)
        n = prob.n
        h = 1.0 / (n - 1)
        g = nm[0]
        x = h * np.arange(n)
        ux = um[2 * g]                                   # [i, j]
        exact = np.outer(np.sin(np.pi * x), np.sin(np.pi * x))
        errs.append(np.abs(ux - exact).max())
        assert np.abs(um[2 * g + 1]).max() <= 5 * errs[-1] + 1e-12
    rates = [np.log2(a / b) / np.log2((2 ** (L + 1) - 1) / (2 ** L - 1)) for a, b, L in zip(errs, errs[1:], (4, 5))]
    assert all(1.8 <= r <= 2.3 for r in rates), (errs, rates)
