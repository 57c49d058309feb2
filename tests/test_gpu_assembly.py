"""GPU assembly (qtt_assemble_stiffness) against the oracle's sparse FEM:
qtt_to_full(K) equals the assembled, masked, concatenated FE matrix to 1e-12
(relative to max |K|), and f likewise, for a single plate, the smooth-load
plate, the L-shaped panel and the two-patch strip."""
import numpy as np
import pytest

import workloads as W
from oracle import fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2501_07778_gb300 as q  # noqa: E402


def _dense(K):
    N = int(np.prod(K.modes))
    return q.qtt_to_full(K).cpu().numpy().reshape(N, N, order="F")


@pytest.mark.parametrize("make,L", [(W.plate_body_force, 3), (W.plate_body_force, 5),
                                    (W.plate_traction_smooth, 4), (W.lshape_shear, 3),
                                    (W.two_patch_strip, 3), (W.lshape_shear, 4)])
def test_assembly_equals_sparse_fem(make, L):
    prob = make(L)
    K, f = q.qtt_assemble_stiffness(prob)
    Kd, fd, _ = fem.duplicated_system(prob)
    Kg = _dense(K)
    scale = np.abs(Kd).max()
    assert np.abs(Kg - Kd.toarray()).max() <= 1e-12 * scale
    fg = q.qtt_to_full(f).cpu().numpy()
    assert np.abs(fg - fd).max() <= 1e-12 * np.abs(fd).max()


def test_assembly_body_force_kinds():
    """All five separable load kinds (1, t, sin, cos, t^2) and a nonzero
    patch offset: compares f with the oracle's consistent load."""
    body = [(0, 1.3, W.SINPI, W.COSPI), (1, -0.7, W.QUAD, W.LIN), (0, 0.4, W.ONE, W.QUAD)]
    prob = W.Problem(L=4, patches=[(0, 0), (1, 0)], E=3.0, nu=0.25,
                     bc=[(W.CLAMP, 0, 0, 0), (0, 0, W.FIX_Y, 0)], body=body,
                     traction=[(1, W.RIGHT, 0.5, -0.25)])
    K, f = q.qtt_assemble_stiffness(prob)
    Kd, fd, _ = fem.duplicated_system(prob)
    fg = q.qtt_to_full(f).cpu().numpy()
    assert np.abs(fg - fd).max() <= 1e-12 * np.abs(fd).max()
    assert np.abs(_dense(K) - Kd.toarray()).max() <= 1e-12 * np.abs(Kd).max()


def test_assembled_ranks_bounded_in_level():
    r6 = max(q.qtt_assemble_stiffness(W.plate_body_force(6))[0].ranks)
    r10 = max(q.qtt_assemble_stiffness(W.plate_body_force(10))[0].ranks)
    assert r10 <= r6 + 2


def test_assembly_rejects_bad_input():
    prob = W.plate_body_force(3)
    prob.bc = [(7, 0, 0, 0)]
    with pytest.raises(q.QttError):
        q.qtt_assemble_stiffness(prob)
