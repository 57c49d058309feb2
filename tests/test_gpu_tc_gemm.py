"""The tcgen05 3xTF32 GEMM (qtt_gemm_tf32x3, through the C ABI) against an
FP64 matrix product of the same FP32 inputs: full tiles, ragged edges in M,
N and K, long K, and a leading dimension that is not a multiple of four."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2501_07778_gb300 as q  # noqa: E402


@pytest.mark.parametrize("M,N,K,pad", [(128, 128, 32, 0), (200, 300, 100, 3), (37, 520, 8, 1), (1000, 64, 3000, 0),
                                       (5, 7, 3, 2), (256, 384, 512, 0)])
def test_tf32x3_gemm_matches_fp64(M, N, K, pad):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K + pad)).astype(np.float32)
    B = rng.standard_normal((N, K + pad)).astype(np.float32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ldd = M + 5
    dD = torch.full((N, ldd), float("nan"), dtype=torch.float32, device="cuda")
    lib = q.lib()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.qtt_gemm_tf32x3(M, N, K, C.c_void_p(dA.data_ptr()), K + pad, C.c_void_p(dB.data_ptr()), K + pad,
                             C.c_void_p(dD.data_ptr()), ldd, s)
    assert rc == 0, lib.qtt_last_error()
    D = dD.cpu().numpy()[:, :M].T.astype(np.float64)
    ref = A[:, :K].astype(np.float64) @ B[:, :K].astype(np.float64).T
    scale = np.abs(A[:, :K]).astype(np.float64) @ np.abs(B[:, :K]).astype(np.float64).T
    assert np.all(np.abs(D - ref) <= 1e-5 * scale + 1e-30), float(np.max(np.abs(D - ref) / scale))
    # the padding columns of D were not written
    assert np.isnan(dD.cpu().numpy()[:, M:]).all()


def _merged_in_qtt_order(prob):
    from oracle import fem
    u, node_map = fem.solve_merged(prob)
    return fem.merged_to_qtt(prob, u, node_map)


@pytest.mark.parametrize("tensor_cores", [1, -1])
def test_mixed_solve_with_tensor_core_local_operator(tensor_cores):
    """QTT_MIXED with the CG forced on every core (local_direct_max = 1): with
    tensor_cores > 0 the FP32 local operator at ranks >= 32 runs as tcgen05
    3xTF32 GEMMs (profile class 10 launches), with < 0 on the SIMT pipes;
    both reach the sparse direct solution."""
    import workloads as W
    lib = q.lib()
    prob = W.plate_top_traction(7, 12.0, 0.28, 1.0, 1.1)
    K, f = q.qtt_assemble_stiffness(prob)
    ms, fl, by, n = C.c_double(), C.c_double(), C.c_double(), C.c_longlong()
    lib.qtt_profile_read(-1, None, None, None, None)
    lib.qtt_profile_enable(1)
    try:
        u, info = q.qtt_solve(K, f, tol=1e-9, precision=q.QTT_MIXED, local_direct_max=1, kick_rank=8,
                              max_sweeps=30, tensor_cores=tensor_cores)
        torch.cuda.synchronize()
    finally:
        lib.qtt_profile_enable(0)
    lib.qtt_profile_read(10, C.byref(ms), C.byref(fl), C.byref(by), C.byref(n))
    lib.qtt_profile_read(-1, None, None, None, None)
    if tensor_cores > 0:
        assert n.value > 0, "the tensor-core GEMM did not run"
    else:
        assert n.value == 0
    ug = q.qtt_to_full(u).cpu().numpy()
    ref = _merged_in_qtt_order(prob)
    err = np.linalg.norm(ug - ref) / np.linalg.norm(ref)
    assert info["rc"] == 0 and info["rel_residual"] <= 1e-9, info
    assert err <= 1e-7, (err, info)


def test_autotuner_times_both_paths_and_solves():
    """tensor_cores = 0: the autotuner times the tensor-core and the SIMT
    operator in every rank bucket it meets and the solve stays exact."""
    import workloads as W
    prob = W.plate_top_traction(8, 40.0, 0.33, 1.3, 2.0)
    K, f = q.qtt_assemble_stiffness(prob)
    for _ in range(2):      # the second solve meets the buckets the first one timed
        u, info = q.qtt_solve(K, f, tol=1e-9, precision=q.QTT_MIXED, local_direct_max=1, kick_rank=8,
                              max_sweeps=30, tensor_cores=0)
        assert info["rc"] == 0 and info["rel_residual"] <= 1e-9, info
    table = q.autotune_table()
    assert table, "no rank bucket reached the autotuner"
    timed = [e for e in table if e["us_tc"] > 0 and e["us_simt"] > 0]
    assert timed, table
    ref = _merged_in_qtt_order(prob)
    ug = q.qtt_to_full(u).cpu().numpy()
    assert np.linalg.norm(ug - ref) / np.linalg.norm(ref) <= 1e-7
