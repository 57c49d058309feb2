"""GB300-native QTT engine for 2D plane-stress elasticity.

Thin Python binding over libqtt.so (include/qtt.h).  The functions carry the
C entry points' names and do argument marshalling only: every step of the
computation runs in the library's CUDA kernels.  Device memory for full
vectors comes from PyTorch; TT cores live in library-owned qtt_tensor
objects wrapped by `QTT`.
"""
from __future__ import annotations

import ctypes as C
import time
from typing import List, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (QTT_F32, QTT_F64, QTT_MIXED, QTT_ORDER_CANONICAL, QTT_ORDER_Z_BLOCK, QttProblem, QttSolveInfo,
                   QttSolveOpts)

__all__ = ["QTT", "QttError", "qtt_assemble_stiffness", "qtt_matvec", "qtt_round", "qtt_solve", "qtt_to_full",
           "qtt_axpby", "qtt_norm", "qtt_residual", "qtt_residual_fe", "qtt_residual_fe_tt", "qtt_fe_apply", "qtt_round_residual", "qtt_to_full_noalloc", "QTT_F64", "QTT_F32", "QTT_MIXED", "QTT_ORDER_Z_BLOCK",
           "QTT_ORDER_CANONICAL", "lib"]


class QttError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.load().qtt_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_lib.ERR_NAMES.get(code, code)}: {msg}")


def lib():
    return _lib.load()


def _check(rc: int, where: str, ok=(0,)):
    if rc not in ok:
        raise QttError(rc, where)
    return rc


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class QTT:
    """Owning handle of a device-resident QTT vector or matrix."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.qtt_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def _info(self):
        L = lib()
        d = C.c_int()
        n = (C.c_int * _lib.QTT_MAX_CORES)()
        m = (C.c_int * _lib.QTT_MAX_CORES)()
        r = (C.c_int * (_lib.QTT_MAX_CORES + 1))()
        p = C.c_int()
        _check(L.qtt_tensor_info(self._h, C.byref(d), n, m, r, C.byref(p)), "qtt_tensor_info")
        dd = d.value
        return dd, list(n[:dd]), list(m[:dd]), list(r[:dd + 1]), p.value

    @property
    def d(self):
        return self._info()[0]

    @property
    def ranks(self) -> List[int]:
        return self._info()[3]

    @property
    def modes(self) -> List[int]:
        return self._info()[1]

    @property
    def col_modes(self) -> List[int]:
        return self._info()[2]

    @property
    def prec(self) -> int:
        return self._info()[4]

    @property
    def is_matrix(self) -> bool:
        return any(x != 1 for x in self.col_modes)

    @classmethod
    def from_cores(cls, cores: Sequence[np.ndarray], prec: int = QTT_F64) -> "QTT":
        """Cores of shape (r0, n, r1) (MPS) or (r0, n, m, r1) (MPO)."""
        d = len(cores)
        dt = np.float64 if prec == QTT_F64 else np.float32
        n = (C.c_int * d)(*[c.shape[1] for c in cores])
        is_mat = cores[0].ndim == 4
        m = (C.c_int * d)(*[(c.shape[2] if is_mat else 1) for c in cores])
        r = (C.c_int * (d + 1))(*([cores[0].shape[0]] + [c.shape[-1] for c in cores]))
        keep = [np.asfortranarray(c, dtype=dt) for c in cores]
        ptrs = (C.c_void_p * d)(*[k.ctypes.data for k in keep])
        h = C.c_void_p()
        _check(lib().qtt_tensor_create(d, n, m if is_mat else None, r, prec, ptrs, C.byref(h)), "qtt_tensor_create")
        return cls(h)

    def cores(self) -> List[np.ndarray]:
        d, n, m, r, p = self._info()
        dt = np.float64 if p == QTT_F64 else np.float32
        is_mat = any(x != 1 for x in m)
        out = []
        for k in range(d):
            shape = (r[k], n[k], m[k], r[k + 1]) if is_mat else (r[k], n[k], r[k + 1])
            out.append(np.empty(shape, dtype=dt, order="F"))
        ptrs = (C.c_void_p * d)(*[o.ctypes.data for o in out])
        _check(lib().qtt_tensor_get_cores(self._h, ptrs), "qtt_tensor_get_cores")
        return out

    def copy(self, prec: Optional[int] = None, stream=None) -> "QTT":
        h = C.c_void_p()
        _check(lib().qtt_tensor_copy(self._h, self.prec if prec is None else prec, C.byref(h), _stream(stream)),
               "qtt_tensor_copy")
        return QTT(h)


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def qtt_to_full(x: QTT, ordering: int = QTT_ORDER_Z_BLOCK, out=None, stream=None):
    """Expand to a full CUDA tensor (torch) of the tensor's precision."""
    import torch
    d, n, m, r, p = x._info()
    total = int(np.prod([a * b for a, b in zip(n, m)], dtype=np.int64))
    dt = torch.float64 if p == QTT_F64 else torch.float32
    if out is None:
        out = torch.empty(total, dtype=dt, device="cuda")
    assert out.is_cuda and out.numel() == total and out.dtype == dt and out.is_contiguous()
    _check(lib().qtt_to_full(x.handle, C.c_void_p(out.data_ptr()), total, ordering, _stream(stream)), "qtt_to_full")
    return out


def qtt_to_full_noalloc(x: QTT, out, stream=None):
    """Z-block expansion of an MPS into the caller's CUDA tensor `out`, with
    the library taking no device memory during the call."""
    import torch
    d, n, m, r, p = x._info()
    total = int(np.prod(n, dtype=np.int64))
    dt = torch.float64 if p == QTT_F64 else torch.float32
    assert out.is_cuda and out.numel() == total and out.dtype == dt and out.is_contiguous()
    _check(lib().qtt_to_full_noalloc(x.handle, C.c_void_p(out.data_ptr()), total, _stream(stream)),
           "qtt_to_full_noalloc")
    return out


def qtt_matvec(A: QTT, x: QTT, tol: float = 0.0, max_rank: int = 0, stream=None) -> QTT:
    h = C.c_void_p()
    _check(lib().qtt_matvec(A.handle, x.handle, tol, max_rank, C.byref(h), _stream(stream)), "qtt_matvec",
           ok=(0, _lib.QTT_ERANKCAP))
    return QTT(h)


def qtt_round(x: QTT, tol: float, max_rank: int = 0, stream=None) -> int:
    return _check(lib().qtt_round(x.handle, tol, max_rank, _stream(stream)), "qtt_round", ok=(0, _lib.QTT_ERANKCAP))


def qtt_axpby(alpha: float, x: QTT, beta: float, y: QTT, stream=None) -> QTT:
    h = C.c_void_p()
    _check(lib().qtt_axpby(alpha, x.handle, beta, y.handle, C.byref(h), _stream(stream)), "qtt_axpby")
    return QTT(h)


def qtt_norm(x: QTT, stream=None) -> float:
    v = C.c_double()
    _check(lib().qtt_norm(x.handle, C.byref(v), _stream(stream)), "qtt_norm")
    return v.value


def qtt_residual(K: QTT, u: QTT, f: QTT, stream=None) -> float:
    v = C.c_double()
    _check(lib().qtt_residual(K.handle, u.handle, f.handle, C.byref(v), _stream(stream)), "qtt_residual")
    return v.value


def qtt_residual_fe(K: QTT, u: QTT, f: QTT, stream=None) -> float:
    """||f - K u|| / ||f|| with K applied as its finite-element stencil."""
    v = C.c_double()
    _check(lib().qtt_residual_fe(K.handle, u.handle, f.handle, C.byref(v), _stream(stream)), "qtt_residual_fe")
    return v.value


def qtt_residual_fe_tt(K: QTT, u: QTT, f: QTT, eps: float = 1e-3, max_rank: int = 128, stream=None):
    """f - K u formed element by element (the FE stencil, FP64) and
    compressed by TT-SVD at relative accuracy eps; returns (r, ||f-Ku||/||f||)."""
    h = C.c_void_p()
    rel = C.c_double()
    _check(lib().qtt_residual_fe_tt(K.handle, u.handle, f.handle, eps, max_rank, C.byref(h), C.byref(rel),
                                    _stream(stream)), "qtt_residual_fe_tt")
    return QTT(h), rel.value


def qtt_fe_apply(K: QTT, x, out=None, stream=None):
    """K x for a full canonical FP64 CUDA tensor x (the assembled FE stencil)."""
    import torch
    assert x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()
    if out is None:
        out = torch.empty_like(x)
    _check(lib().qtt_fe_apply(K.handle, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), x.numel(),
                              _stream(stream)), "qtt_fe_apply")
    return out


def qtt_round_residual(K: QTT, u: QTT, f: QTT, rank: int, seed: int = 0, stream=None):
    """Randomized rank-`rank` FP64 rounding of f - K u; returns (r, ||r||)."""
    h = C.c_void_p()
    kept = C.c_double()
    _check(lib().qtt_round_residual(K.handle, u.handle, f.handle, rank, seed, C.byref(kept), C.byref(h),
                                    _stream(stream)), "qtt_round_residual")
    return QTT(h), kept.value


def autotune_table():
    """The autotuner's decisions on this device: list of dicts (rank buckets,
    microseconds per Krylov iteration on tensor cores and SIMT)."""
    n = C.c_int()
    lib().qtt_autotune_table(0, C.byref(n), None, None, None, None)
    k = n.value
    b0, b1 = (C.c_int * max(1, k))(), (C.c_int * max(1, k))()
    tc, sm = (C.c_double * max(1, k))(), (C.c_double * max(1, k))()
    lib().qtt_autotune_table(k, C.byref(n), b0, b1, tc, sm)
    return [{"r0_bucket": b0[i], "r1_bucket": b1[i], "us_tc": tc[i], "us_simt": sm[i],
             "choice": ("tc" if 0 <= tc[i] < sm[i] else "simt") if tc[i] >= 0 and sm[i] >= 0 else "timing"}
            for i in range(k)]


def make_problem_struct(prob, tol: float = 0.0):
    """Marshal a workloads.Problem into the C struct (arrays kept alive on the
    returned struct)."""
    q = prob.q
    patch = (C.c_int * (2 * q))(*[v for xy in prob.patches for v in xy])
    bc = (C.c_int * (4 * q))(*[v for sides in prob.bc for v in sides])
    nb = len(prob.body)
    bt = (C.c_int * max(1, 3 * nb))(*[v for (c, a, kx, ky) in prob.body for v in (c, kx, ky)])
    bcf = (C.c_double * max(1, nb))(*[a for (c, a, kx, ky) in prob.body])
    nt = len(prob.traction)
    tw = (C.c_int * max(1, 2 * nt))(*[v for (m, s, tx, ty) in prob.traction for v in (m, s)])
    tv = (C.c_double * max(1, 2 * nt))(*[v for (m, s, tx, ty) in prob.traction for v in (tx, ty)])
    dirs = getattr(prob, "dirichlet", []) or []
    nd = len(dirs)
    dt = (C.c_int * max(1, 3 * nd))(*[v for (c, a, kx, ky) in dirs for v in (c, kx, ky)])
    dcf = (C.c_double * max(1, nd))(*[a for (c, a, kx, ky) in dirs])
    st = QttProblem(prob.L, q, patch, prob.E, prob.nu, bc, nb, bt, bcf, nt, tw, tv, prob.gamma, tol, nd, dt, dcf)
    st._keep = (patch, bc, bt, bcf, tw, tv, dt, dcf)
    return st


def qtt_assemble_stiffness(prob, tol: float = 0.0, stream=None):
    """Assemble (K, f) of a workloads.Problem on the device (Algorithm 1)."""
    st = make_problem_struct(prob, tol)
    hK, hf = C.c_void_p(), C.c_void_p()
    _check(lib().qtt_assemble_stiffness(C.byref(st), C.byref(hK), C.byref(hf), _stream(stream)),
           "qtt_assemble_stiffness")
    return QTT(hK), QTT(hf)


def solve_opts(tol=1e-8, max_rank=0, kick_rank=0, max_sweeps=0, local_direct_max=0, local_restart=0,
               local_max_cycles=0, precision=QTT_F64, refine_max=0, inner_tol=0.0, verbose=0,
               tensor_cores=0) -> QttSolveOpts:
    return QttSolveOpts(tol, max_rank, kick_rank, max_sweeps, local_direct_max, local_restart, local_max_cycles,
                        precision, refine_max, inner_tol, verbose, tensor_cores)


def qtt_solve_batched(Ks: List[QTT], fs: List[QTT], x0s: Optional[List[Optional[QTT]]] = None, nworkers: int = 0,
                      stream=None, **opts):
    """Solve independent problems together; returns (list of u, list of info dicts)."""
    n = len(Ks)
    o = solve_opts(**opts)
    Karr = (C.c_void_p * n)(*[k.handle for k in Ks])
    farr = (C.c_void_p * n)(*[f.handle for f in fs])
    xarr = None
    if x0s is not None:
        xarr = (C.c_void_p * n)(*[(x.handle if x is not None else None) for x in x0s])
    out = (C.c_void_p * n)()
    infos = (QttSolveInfo * n)()
    rc = lib().qtt_solve_batched(n, Karr, farr, xarr, C.byref(o), nworkers, out, infos, _stream(stream))
    _check(rc, "qtt_solve_batched", ok=(0, _lib.QTT_ENOCONV))
    us = [QTT(C.c_void_p(out[i])) if out[i] else None for i in range(n)]
    ds = [{k: getattr(infos[i], k) for k, _ in QttSolveInfo._fields_} for i in range(n)]
    return us, ds


def qtt_solve(K: QTT, f: QTT, x0: Optional[QTT] = None, z0: Optional[QTT] = None, stream=None, check=True,
              **opts):
    """Solve K u = f by AMEn; returns (u, info dict)."""
    o = solve_opts(**opts)
    info = QttSolveInfo()
    h = C.c_void_p()
    rc = lib().qtt_solve(K.handle, f.handle, x0.handle if x0 is not None else None,
                         z0.handle if z0 is not None else None, C.byref(o), C.byref(h), C.byref(info),
                         _stream(stream))
    if check:
        _check(rc, "qtt_solve", ok=(0, _lib.QTT_ENOCONV))
    d = {k: getattr(info, k) for k, _ in QttSolveInfo._fields_}
    d["rc"] = rc
    return (QTT(h) if h.value else None), d
