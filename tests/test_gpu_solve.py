"""GPU AMEn solve (qtt_solve) against the oracle: the full displacement
vector against the sparse direct FE solution (relative L2 <= 1e-8 in FP64 at
tolerance 1e-10), the oracle's own AMEn on the same inputs, the multi-patch
concatenated system, and mixed precision with FP64 refinement."""
import numpy as np
import pytest

import workloads as W
from oracle import amen, assembly, fem, tt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2501_07778_gb300 as q  # noqa: E402


def _x0z0(prob, rx=2, rz=4, seed=5):
    modes = W.qtt_modes(prob)
    x0 = W.random_tt(seed, modes, [1] + [rx] * (len(modes) - 1) + [1])
    z0 = W.random_tt(seed + 1, modes, [1] + [rz] * (len(modes) - 1) + [1])
    return x0, z0


@pytest.mark.parametrize("make,L", [(W.plate_body_force, 3), (W.plate_body_force, 5), (W.lshape_shear, 3)])
def test_solve_matches_sparse_direct(make, L):
    prob = make(L)
    K, f = q.qtt_assemble_stiffness(prob)
    x0, z0 = _x0z0(prob)
    u, info = q.qtt_solve(K, f, q.QTT.from_cores(x0), q.QTT.from_cores(z0), tol=1e-10, max_sweeps=40)
    assert info["rc"] == 0, info
    ug = q.qtt_to_full(u).cpu().numpy()
    ref = fem.solve_duplicated(prob)
    err = np.linalg.norm(ug - ref) / np.linalg.norm(ref)
    assert err <= 1e-8, (err, info)
    assert info["rel_residual"] <= 1e-8


def test_solve_matches_oracle_amen():
    prob = W.plate_traction_smooth(4)
    Ko, fo = assembly.assemble(prob)
    x0, z0 = _x0z0(prob)
    xo, io = amen.amen_solve(Ko, fo, x0, z0, 1e-9, max_sweeps=30, local_direct_max=2048)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, q.QTT.from_cores(x0), q.QTT.from_cores(z0), tol=1e-9, max_sweeps=30,
                          local_direct_max=2048)
    assert info["rc"] == 0 and io.converged
    ug = q.qtt_to_full(u).cpu().numpy()
    uo = tt.full(xo)
    assert np.linalg.norm(ug - uo) / np.linalg.norm(uo) <= 1e-7


def test_solve_gmres_path():
    """Force the iterative local solver (dense LU disabled)."""
    prob = W.plate_body_force(4)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-9, max_sweeps=40, local_direct_max=1, local_restart=40,
                          local_max_cycles=20)
    ug = q.qtt_to_full(u).cpu().numpy()
    ref = fem.solve_duplicated(prob)
    err = np.linalg.norm(ug - ref) / np.linalg.norm(ref)
    assert err <= 1e-6, (err, info)


def test_solve_mixed_precision_refinement():
    prob = W.plate_body_force(5)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-9, precision=q.QTT_MIXED, inner_tol=1e-4, refine_max=8, max_sweeps=30)
    ug = q.qtt_to_full(u).cpu().numpy()
    ref = fem.solve_duplicated(prob)
    err = np.linalg.norm(ug - ref) / np.linalg.norm(ref)
    assert info["rc"] == 0, info
    assert info["rel_residual"] <= 1e-9
    assert err <= 1e-7, (err, info)


def test_batched_uneven_problems_match_oracle():
    """Uneven batch (levels 3-5, one to three patches) through the work queue
    with several concurrent workers: every result matches its own sparse
    direct solution."""
    probs = [W.plate_body_force(4), W.lshape_shear(3), W.two_patch_strip(4), W.plate_traction_smooth(5),
             W.plate_top_traction(3, 20.0, 0.35, 1.5, 1.0)]
    KF = [q.qtt_assemble_stiffness(p) for p in probs]
    us, infos = q.qtt_solve_batched([k for k, _ in KF], [f for _, f in KF], nworkers=3, tol=1e-10, max_sweeps=40)
    torch.cuda.synchronize()
    for p, u, info in zip(probs, us, infos):
        assert info["status"] == 0, info
        ug = q.qtt_to_full(u).cpu().numpy()
        ref = fem.solve_duplicated(p)
        assert np.linalg.norm(ug - ref) / np.linalg.norm(ref) <= 1e-8


def _oracle_residual(prob, u_cores):
    Ko, fo = assembly.assemble(prob)
    return tt.full(fo) - tt.full_matrix(Ko) @ tt.full(u_cores)


def test_round_residual_full_rank_is_exact():
    """At a sketch rank that reaches the ranks of f - K u, the randomized
    rounding returns the residual itself (oracle: dense f - K u)."""
    prob = W.plate_body_force(3)
    K, f = q.qtt_assemble_stiffness(prob)
    uc = W.random_tt(21, W.qtt_modes(prob), [1, 3, 5, 4, 1])
    r, kept = q.qtt_round_residual(K, q.QTT.from_cores(uc), f, rank=512, seed=3)
    ro = _oracle_residual(prob, uc)
    rg = q.qtt_to_full(r).cpu().numpy()
    assert np.linalg.norm(rg - ro) <= 1e-11 * np.linalg.norm(ro)
    assert abs(kept - np.linalg.norm(ro)) <= 1e-11 * np.linalg.norm(ro)


@pytest.mark.parametrize("rank", [4, 12, 40])
def test_round_residual_is_orthogonal_projection(rank):
    """||r - r~||^2 + ||r~||^2 = ||r||^2 at any sketch rank, the error shrinks
    as the rank grows, and the cores come back left-orthonormal."""
    prob = W.plate_traction_smooth(5)
    K, f = q.qtt_assemble_stiffness(prob)
    uc = W.random_tt(22, W.qtt_modes(prob), [1, 4, 6, 6, 6, 4, 1])
    r, kept = q.qtt_round_residual(K, q.QTT.from_cores(uc), f, rank=rank, seed=7)
    ro = _oracle_residual(prob, uc)
    rg = q.qtt_to_full(r).cpu().numpy()
    nr, ne = np.linalg.norm(ro), np.linalg.norm(ro - rg)
    assert abs(kept - np.linalg.norm(rg)) <= 1e-12 * nr
    assert abs(ne ** 2 + kept ** 2 - nr ** 2) <= 1e-10 * nr ** 2
    cores = r.cores()
    for c in cores[:-1]:
        m = c.reshape(-1, c.shape[-1], order="F")
        np.testing.assert_allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-12)
    if rank == 40:
        # the sketch reaches at least the TT-SVD of the same rank within a small factor
        best = tt.tt_svd(ro, W.qtt_modes(prob), 0.0, max_rank=rank)
        assert ne <= 5.0 * np.linalg.norm(ro - tt.full(best)) + 1e-12 * nr


@pytest.mark.parametrize("precision", [q.QTT_F64, q.QTT_MIXED])
def test_refinement_recovers_truncated_sweeps(precision):
    """Sweeps cut short (five sweeps, slow rank growth) leave the first
    iterate far above tol; the outer refinement (randomized FP64 residual,
    correction solve, u + d) must still reach the sparse direct solution."""
    prob = W.plate_body_force(5)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-9, precision=precision, kick_rank=4, max_sweeps=5, refine_max=12)
    ug = q.qtt_to_full(u).cpu().numpy()
    ref = fem.solve_duplicated(prob)
    err = np.linalg.norm(ug - ref) / np.linalg.norm(ref)
    assert info["refinements"] >= 1, info
    assert info["rc"] == 0 and info["rel_residual"] <= 1e-9, info
    assert err <= 1e-7, (err, info)
