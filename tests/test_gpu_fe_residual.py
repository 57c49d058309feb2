"""qtt_residual_fe (K applied as its finite-element stencil in full format)
against the oracle's assembled systems and against the exact QTT route
(qtt_residual), for one patch and for concatenated multi-patch systems, at
residuals of order one (random u) and near the solution."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, stencil

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2501_07778_gb300 as q  # noqa: E402
from paper_2501_07778_gb300 import _lib  # noqa: E402

PROBLEMS = [(W.plate_top_traction, (5, 30.0, 0.31, 1.2, 0.4)), (W.plate_body_force, (4,)),
            (W.two_patch_strip, (4,)), (W.lshape_shear, (5,)), (W.plate_traction_smooth, (6,))]


def _oracle_rel(prob, u_qtt_order):
    K, f, _ = fem.duplicated_system(prob, masked=True)
    r = f - K @ u_qtt_order
    return np.linalg.norm(r) / np.linalg.norm(f)


@pytest.mark.parametrize("make,args", PROBLEMS)
def test_fe_residual_matches_oracle_system_random_u(make, args):
    prob = make(*args)
    K, f = q.qtt_assemble_stiffness(prob)
    uc = W.random_tt(41, W.qtt_modes(prob), [1] + [3] * (len(W.qtt_modes(prob)) - 1) + [1])
    u = q.QTT.from_cores(uc)
    got = q.qtt_residual_fe(K, u, f)
    ug = q.qtt_to_full(u).cpu().numpy()
    want = _oracle_rel(prob, ug)
    assert abs(got - want) <= 1e-11 * want, (got, want)
    exact_qtt = q.qtt_residual(K, u, f)
    assert abs(got - exact_qtt) <= 1e-10 * exact_qtt, (got, exact_qtt)


@pytest.mark.parametrize("make,args", PROBLEMS)
def test_fe_residual_near_the_solution(make, args):
    """At a converged solve the three residuals (GPU stencil, oracle sparse
    system, exact QTT product of the rounded K) agree far below the 1e-8
    acceptance level."""
    prob = make(*args)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-10, max_sweeps=40)
    got = q.qtt_residual_fe(K, u, f)
    want = _oracle_rel(prob, q.qtt_to_full(u).cpu().numpy())
    exact_qtt = q.qtt_residual(K, u, f)
    assert got <= 1e-9 and want <= 1e-9
    # the stencil is the oracle's finite-element system exactly ...
    assert abs(got - want) <= 1e-11, (got, want)
    # ... while the QTT product uses K as rounded by the assembly (tolerance
    # 1e-13 relative); the difference stays two orders below acceptance (1e-8)
    assert abs(got - exact_qtt) <= 1e-10, (got, exact_qtt)


def test_fe_residual_one_patch_matches_host_stencil_L8():
    prob = W.plate_top_traction(8, 3.0, 0.4, 1.0, 2.2)
    K, f = q.qtt_assemble_stiffness(prob)
    modes = W.qtt_modes(prob)
    uc = W.random_tt(42, modes, [1] + [6] * (len(modes) - 1) + [1], scale=1e-2)
    u = q.QTT.from_cores(uc)
    got = q.qtt_residual_fe(K, u, f)
    uf = q.qtt_to_full(u, ordering=q.QTT_ORDER_CANONICAL).cpu().numpy()
    r, fbc = stencil.masked_residual(prob, uf)
    want = np.linalg.norm(r) / np.linalg.norm(fbc)
    assert abs(got - want) <= 1e-11 * want, (got, want)


def test_fe_residual_refuses_a_rounded_operator():
    prob = W.plate_body_force(4)
    K, f = q.qtt_assemble_stiffness(prob)
    u = q.QTT.from_cores(W.random_tt(43, W.qtt_modes(prob), [1, 2, 2, 2, 2, 1]))
    q.qtt_residual_fe(K, u, f)
    q.qtt_round(K, 1e-14)
    with pytest.raises(q.QttError) as e:
        q.qtt_residual_fe(K, u, f)
    assert e.value.code == _lib.QTT_EINVAL


@pytest.mark.parametrize("make,args", PROBLEMS)
def test_fe_residual_tt_matches_oracle_vector(make, args):
    """qtt_residual_fe_tt: the QTT residual expanded back equals the oracle's
    f - K u (masked duplicated system, QTT order) within the TT-SVD bound
    eps ||r||, its ranks respect the cap, and rel is the stencil residual."""
    prob = make(*args)
    K, f = q.qtt_assemble_stiffness(prob)
    modes = W.qtt_modes(prob)
    u = q.QTT.from_cores(W.random_tt(44, modes, [1] + [4] * (len(modes) - 1) + [1]))
    Ko, fo, _ = fem.duplicated_system(prob, masked=True)
    r_or = fo - Ko @ q.qtt_to_full(u).cpu().numpy()
    eps = 1e-5
    r, rel = q.qtt_residual_fe_tt(K, u, f, eps=eps, max_rank=512)
    got = q.qtt_to_full(r).cpu().numpy()
    assert np.linalg.norm(got - r_or) <= 2 * eps * np.linalg.norm(r_or)
    assert abs(rel - np.linalg.norm(r_or) / np.linalg.norm(fo)) <= 1e-11 * rel
    r4, _ = q.qtt_residual_fe_tt(K, u, f, eps=eps, max_rank=4)
    assert max(r4.ranks) <= 4


def test_fe_residual_tt_keeps_the_error_carrying_part():
    """Near the solution the residual is dominated by high-frequency parts
    whose image under K^-1 is small; the compressed residual at eps = 1e-3
    must keep K^-1 r (what an outer correction solves for) to within 5 %."""
    import scipy.sparse.linalg as spla
    prob = W.plate_traction_smooth(6)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-9, max_sweeps=30, refine_max=-1)
    Ko, fo, _ = fem.duplicated_system(prob, masked=True)
    lu = spla.splu(Ko.tocsc())
    r_or = fo - Ko @ q.qtt_to_full(u).cpu().numpy()
    r, _ = q.qtt_residual_fe_tt(K, u, f, eps=1e-3, max_rank=128)
    e_or = lu.solve(r_or)
    e_tt = lu.solve(q.qtt_to_full(r).cpu().numpy())
    assert np.linalg.norm(e_tt - e_or) <= 0.05 * np.linalg.norm(e_or)
