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
