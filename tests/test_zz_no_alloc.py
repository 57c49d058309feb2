"""The allocation-free Z-block expansion (qtt_to_full_noalloc, through the C
ABI) against the oracle's entry-wise expansion and against the ordinary
qtt_to_full on the same tensors, two calls in a row; that the calls take no
device memory; and its argument and size checks.  Collected last on purpose:
the first call on a device sets up the fixed scratch buffer."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import tt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2501_07778_gb300 as q  # noqa: E402
from paper_2501_07778_gb300 import _lib  # noqa: E402

CASES = [
    ([4, 4, 4, 2], [1, 3, 7, 2, 1], q.QTT_F64),
    ([4] * 8 + [3, 2], [1, 4, 16, 37, 70, 61, 33, 17, 6, 2, 1], q.QTT_F64),
    ([4] * 9 + [2], [1, 4, 16, 29, 45, 45, 30, 16, 8, 2, 1], q.QTT_F32),
    ([5], [1, 1], q.QTT_F64),
]


@pytest.mark.parametrize("modes,ranks,prec", CASES)
def test_noalloc_matches_oracle_and_to_full_twice(modes, ranks, prec):
    cores = W.random_tt(11, modes, ranks)
    x = q.QTT.from_cores(cores, prec)
    # the oracle expands the cores the library actually holds (FP32 cases
    # are rounded on upload)
    want = tt.full([np.asarray(c, dtype=np.float64) for c in x.cores()])
    ref = q.qtt_to_full(x)
    tol = 1e-13 if prec == q.QTT_F64 else 1e-5
    scale = float(np.abs(want).max())
    lib = _lib.load()
    out = torch.full_like(ref, float("nan"))
    q.qtt_to_full_noalloc(x, out)          # the first call may set up the buffer
    torch.cuda.synchronize()
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        allocs = lib.qtt_device_allocations()
        q.qtt_to_full_noalloc(x, out)
        torch.cuda.synchronize()
        assert lib.qtt_device_allocations() == allocs, "qtt_to_full_noalloc took device memory"
        got = out.double().cpu().numpy()
        assert float(np.abs(got - want).max()) <= tol * scale
        assert float((out - ref).abs().max()) <= tol * scale


def test_noalloc_rejects_oversized_and_mpo():
    lib = _lib.load()
    # partial expansions of this 12-core tensor take about 41 MiB (> 32 MiB)
    modes = [4] * 12
    ranks = [1, 4, 16, 64, 256, 512, 512, 512, 256, 64, 16, 4, 1]
    x = q.QTT.from_cores(W.random_tt(12, modes, ranks))
    total = 4 ** 12
    out = torch.empty(total, dtype=torch.float64, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.qtt_to_full_noalloc(x.handle, C.c_void_p(out.data_ptr()), total, s)
    assert rc == _lib.QTT_EINVAL
    assert b"scratch" in lib.qtt_last_error()
    # size mismatch
    rc = lib.qtt_to_full_noalloc(x.handle, C.c_void_p(out.data_ptr()), total - 1, s)
    assert rc == _lib.QTT_EINVAL
    # MPO
    A = q.QTT.from_cores(W.random_mpo(3, [4, 2], [4, 2], [1, 3, 1]))
    buf = torch.empty(64, dtype=torch.float64, device="cuda")
    rc = lib.qtt_to_full_noalloc(A.handle, C.c_void_p(buf.data_ptr()), 8, s)
    assert rc == _lib.QTT_EINVAL
    # the library still works afterwards
    cores = W.random_tt(4, [4, 4, 2], [1, 3, 2, 1])
    y = q.QTT.from_cores(cores)
    o = torch.empty(32, dtype=torch.float64, device="cuda")
    q.qtt_to_full_noalloc(y, o)
    np.testing.assert_allclose(o.cpu().numpy(), tt.full(cores), rtol=1e-13, atol=1e-14)
