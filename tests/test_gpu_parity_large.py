"""GPU parity on the code paths the solver takes at full size.

* qtt_round_residual against the oracle's randomized rounding (O-4) entry by
  entry, with the same cores, seed and sketch ranks;
* the persistent FP32 local CG of QTT_MIXED (forced by local_direct_max = 1,
  its launches counted by the event profiler) against sparse direct;
* the three-patch L-shape in QTT_MIXED with refinement against sparse
  direct;
* the L = 10 plate with traction and smooth body force in FP64 at tolerance
  1e-10 against sparse direct (full displacement vector);
* the L = 12 bench workload solved exactly as the benchmark solves it, its
  residual recomputed on the host by the matrix-free FP64 stencil (O-3).
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import fem, randround, stencil, tt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2501_07778_gb300 as q  # noqa: E402


def _merged_in_qtt_order(prob):
    u, node_map = fem.solve_merged(prob)
    return fem.merged_to_qtt(prob, u, node_map)


@pytest.mark.parametrize("ell", [4, 12, 40])
def test_round_residual_matches_oracle_entry_by_entry(ell):
    modes = [4, 4, 4, 4, 3, 2]
    Kc = W.random_mpo(31, modes, modes, [1, 3, 5, 6, 5, 3, 1])
    uc = W.random_tt(32, modes, [1, 4, 7, 9, 6, 2, 1])
    fc = W.random_tt(33, modes, [1, 2, 3, 3, 2, 2, 1])
    seed = 0x5eed0000 + ell
    ro, no = randround.round_residual(Kc, uc, fc, ell=ell, seed=seed)
    r, kept = q.qtt_round_residual(q.QTT.from_cores(Kc), q.QTT.from_cores(uc), q.QTT.from_cores(fc), rank=ell,
                                   seed=seed)
    assert r.ranks == tt.ranks(ro)
    want = tt.full(ro)
    got = q.qtt_to_full(r).cpu().numpy()
    scale = np.linalg.norm(tt.full(randround.residual_tt(Kc, uc, fc)))
    assert np.abs(got - want).max() <= 1e-12 * scale
    assert abs(kept - no) <= 1e-12 * scale


def test_mixed_persistent_cg_path_matches_sparse_direct():
    lib = q.lib()
    prob = W.plate_top_traction(6, 40.0, 0.3, 1.0, 0.7)
    K, f = q.qtt_assemble_stiffness(prob)
    ms, fl, by, n = C.c_double(), C.c_double(), C.c_double(), C.c_longlong()
    lib.qtt_profile_read(-1, C.byref(ms), C.byref(fl), C.byref(by), C.byref(n))
    lib.qtt_profile_enable(1)
    try:
        u, info = q.qtt_solve(K, f, tol=1e-9, precision=q.QTT_MIXED, local_direct_max=1, kick_rank=8,
                              max_sweeps=30)
        torch.cuda.synchronize()
    finally:
        lib.qtt_profile_enable(0)
    lib.qtt_profile_read(8, C.byref(ms), C.byref(fl), C.byref(by), C.byref(n))
    lib.qtt_profile_read(-1, None, None, None, None)
    assert n.value > 0, "the persistent FP32 CG kernel did not run"
    ug = q.qtt_to_full(u).cpu().numpy()
    ref = _merged_in_qtt_order(prob)
    err = np.linalg.norm(ug - ref) / np.linalg.norm(ref)
    assert info["rc"] == 0 and info["rel_residual"] <= 1e-9, info
    assert err <= 1e-7, (err, info)


def test_lshape_mixed_refinement_matches_sparse_direct():
    prob = W.lshape_shear(6)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-9, precision=q.QTT_MIXED, kick_rank=8, max_sweeps=30, refine_max=8)
    ug = q.qtt_to_full(u).cpu().numpy()
    ref = fem.solve_duplicated(prob)
    err = np.linalg.norm(ug - ref) / np.linalg.norm(ref)
    assert info["rc"] == 0 and info["rel_residual"] <= 1e-9, info
    assert err <= 1e-7, (err, info)


def test_config2_plate_L10_fp64_full_vector():
    """Plate at L = 10 (2.1 M DOFs), right-edge traction (1, 0) and body
    force (sin(pi x) sin(pi y), x y), FP64 at tolerance 1e-10: relative L2
    error of the whole displacement vector against sparse direct <= 1e-8."""
    prob = W.plate_traction_smooth(10)
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-10, precision=q.QTT_F64, kick_rank=8, max_sweeps=24)
    ug = q.qtt_to_full(u).cpu().numpy()
    del u
    ref = _merged_in_qtt_order(prob)
    err = np.linalg.norm(ug - ref) / np.linalg.norm(ref)
    assert info["rel_residual"] <= 1e-9, info
    assert err <= 1e-8, (err, info)


def test_bench_workload_L12_residual_by_host_stencil():
    """The L = 12 plate of the benchmark (33.5 M DOFs), solved with the
    benchmark's options; the FP64 residual f - K u of the expanded solution,
    recomputed on the host element by element, is <= 1e-8 of ||f||."""
    E, nu, amp, th = W.plate_params(2, 1)[0]
    prob = W.plate_top_traction(12, float(E), float(nu), float(amp), float(th))
    K, f = q.qtt_assemble_stiffness(prob)
    u, info = q.qtt_solve(K, f, tol=1e-8, precision=q.QTT_MIXED, kick_rank=8, max_sweeps=24)
    assert info["rc"] == 0 and info["rel_residual"] <= 1e-8, info
    ug = q.qtt_to_full(u, ordering=q.QTT_ORDER_CANONICAL).cpu().numpy()
    del u, K, f
    r, fbc = stencil.masked_residual(prob, ug)
    rel = np.linalg.norm(r) / np.linalg.norm(fbc)
    assert rel <= 1e-8, (rel, info)
