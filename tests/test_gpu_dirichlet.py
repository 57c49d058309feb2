"""Nonhomogeneous Dirichlet data (Algorithm 1's u0) on the GPU: the lifted
load f = M (f - K g) + g against the oracle's masked duplicated system, the
patch test (a linear u0 on every outer side with no load is reproduced
exactly, one patch and the L-shape) and a prescribed nonzero edge against
sparse direct."""
import numpy as np
import pytest

import workloads as W
from oracle import fem, indexing

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2501_07778_gb300 as q  # noqa: E402


@pytest.mark.parametrize("prob", [W.patch_test(4), W.patch_test(3, ((0, 0), (1, 0), (0, 1))),
                                  W.plate_prescribed_edge(4)])
def test_lifted_assembly_equals_oracle(prob):
    K, f = q.qtt_assemble_stiffness(prob)
    Kd, fd, _ = fem.duplicated_system(prob)
    N = int(np.prod(K.modes))
    Kg = q.qtt_to_full(K).cpu().numpy().reshape(N, N, order="F")
    assert np.abs(Kg - Kd.toarray()).max() <= 1e-12 * np.abs(Kd).max()
    fg = q.qtt_to_full(f).cpu().numpy()
    assert np.abs(fg - fd).max() <= 1e-12 * np.abs(fd).max()


@pytest.mark.parametrize("patches,L", [(((0, 0),), 6), (((0, 0), (1, 0), (0, 1)), 5)])
def test_patch_test_reproduces_linear_field(patches, L):
    prob = W.patch_test(L, patches)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-11, max_sweeps=30)
    ug = q.qtt_to_full(u).cpu().numpy()
    n, nq = prob.n, prob.q
    nn = n * n
    h = 1.0 / (n - 1)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    z = indexing.zorder(ii, jj, L)
    for m, (ox, oy) in enumerate(prob.patches):
        x, y = ox + h * ii, oy + h * jj
        ux = ug[(z + nn * m).ravel()]
        uy = ug[(z + nn * m + nn * nq).ravel()]
        assert np.abs(ux - (0.1 + 0.2 * x - 0.3 * y).ravel()).max() <= 1e-8, info
        assert np.abs(uy - (-0.05 + 0.1 * x + 0.25 * y).ravel()).max() <= 1e-8, info


def test_prescribed_edge_matches_sparse_direct():
    prob = W.plate_prescribed_edge(6)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-10, precision=q.QTT_MIXED, kick_rank=8, max_sweeps=30)
    ug = q.qtt_to_full(u).cpu().numpy()
    um, nm = fem.solve_merged(prob)
    ref = fem.merged_to_qtt(prob, um, nm)
    err = np.linalg.norm(ug - ref) / np.linalg.norm(ref)
    assert info["rc"] == 0 and info["rel_residual"] <= 1e-10, info
    assert err <= 1e-8, (err, info)
