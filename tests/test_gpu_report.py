"""The Section 5 level study (paper_2501_07778_gb300.report): errors against
the self-refined reference fall at the Q1 orders (h^2 in L2, h in the
energy seminorm), the parameter counts and ranks are those of the returned
cores, the effective rank is the oracle's for the same cores, and the FE
operator apply used for the energy norm matches the oracle's sparse system."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, tt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2501_07778_gb300 as q  # noqa: E402
from paper_2501_07778_gb300 import report  # noqa: E402


def _canonical_to_qtt(prob):
    """index map: position in QTT order of every canonical DOF"""
    from oracle import indexing
    n, nq, L = prob.n, prob.q, prob.L
    nn = n * n
    m, j, i, c = np.meshgrid(np.arange(nq), np.arange(n), np.arange(n), np.arange(2), indexing="ij")
    return (indexing.zorder(i, j, L) + nn * m + nn * nq * c).ravel()


@pytest.mark.parametrize("make,L", [(W.plate_traction_smooth, 4), (W.lshape_shear, 4), (W.patch_test, 3)])
def test_fe_apply_matches_oracle_system(make, L):
    """qtt_fe_apply on a full canonical vector equals the oracle's masked,
    concatenated sparse matrix times the same vector (element by element)."""
    prob = make(L)
    K, f = q.qtt_assemble_stiffness(prob)
    Kd, _, _ = fem.duplicated_system(prob)
    perm = _canonical_to_qtt(prob)
    x = np.random.default_rng(L).standard_normal(perm.size)
    xq = np.empty_like(x)
    xq[perm] = x
    y = q.qtt_fe_apply(K, torch.from_numpy(x).cuda()).cpu().numpy()
    want = (Kd @ xq)[perm]
    assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max()


def test_level_study_orders_and_counts():
    """Smooth manufactured solution (fully clamped plate): the field error
    falls as h^2 in L2 and h in energy (Q1); a clamped-free corner (the
    cantilever plates) lowers both."""
    recs = report.study(W.plate_manufactured, [4, 5, 6, 7], ref_level=10, tol=1e-10)
    lv = [r for r in recs if "err_l2" in r]
    e2 = [r["err_l2"] for r in lv]
    ee = [r["err_energy"] for r in lv]
    assert all(a > b for a, b in zip(e2, e2[1:])) and all(a > b for a, b in zip(ee, ee[1:]))
    rt = report.rates(recs)
    assert 1.7 <= rt["order_err_l2"] <= 2.3, rt
    assert 0.8 <= rt["order_err_energy"] <= 1.2, rt
    # the nodal difference to the interpolated reference is superconvergent
    # on uniform Q1 meshes: O(h^2) in the discrete energy norm as well
    assert 1.7 <= rt["order_err_l2_nodal"] <= 2.3, rt
    assert 1.7 <= rt["order_err_energy_nodal"] <= 2.3, rt
    for r in recs:
        ranks = r["ranks"]
        assert r["R_d"] == max(ranks)
        # (the reference level may stop a little above its 1e-10 target in
        # mixed precision; its residual stays far below the errors measured)
        assert r["rel_residual"] <= 1e-8, r
    # effective rank and N_d of a solution against the oracle's definitions
    prob = W.plate_traction_smooth(6)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-10)
    cores = u.cores()
    assert abs(info["erank"] - tt.erank(cores)) <= 1e-9 * tt.erank(cores)
    assert sum(c.size for c in cores) == tt.n_params(cores)
