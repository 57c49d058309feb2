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
