"""Level study of Section 5: compression and convergence of the QTT solution
as the mesh is refined.

For a problem family and a range of levels d (n = 2^d nodes per patch side)
every record holds what the paper plots against d:
  * the solution's QTT ranks, R_d = max_k r_k, its parameter count N_d =
    sum_k r_{k-1} n_k r_k and effective rank (Section 4);
  * the memory of the assembled K and f and of the solution (FP64 cores);
  * the solve's time, sweeps and FP64 relative residual;
  * the error against a self-refined reference, the solution at the finest
    level ref_level: the coarse Q1 field prolonged (bilinear on each patch)
    to the reference mesh, e = u_ref - P u_h, in the relative L2 norm and
    the energy seminorm sqrt(e^T K e / u_ref^T K u_ref) of the reference
    mesh (err_l2, err_energy: the errors of the field, O(h^2) and O(h) for
    smooth solutions); and the nodal difference u_h - I u_ref on the coarse
    mesh (err_l2_nodal, err_energy_nodal: superconvergent, O(h^2) in both on
    these uniform meshes).  Operators are applied by qtt_fe_apply.
`rates` fits the algebraic order of the errors in h and the exponential
rate of the error in N_d.  Every number comes from the library's kernels;
the interpolation and the norms are elementwise device tensor operations.
"""
from __future__ import annotations

import math
import time
from typing import Callable, Dict, List

import numpy as np

from . import QTT_MIXED, QTT_ORDER_CANONICAL, qtt_assemble_stiffness, qtt_fe_apply, qtt_solve, qtt_to_full


def _bytes(t) -> int:
    d, n, m, r, p = t._info()
    return sum(r[k] * n[k] * m[k] * r[k + 1] for k in range(d)) * (8 if p == 0 else 4)


def _grid(u_can, q: int, n: int):
    """Canonical full vector -> tensor [patch, component, j, i]."""
    return u_can.view(q, n, n, 2).permute(0, 3, 1, 2)


def interpolate(u_src, q: int, L_src: int, L_dst: int):
    """The Q1 field of a canonical vector on the level-L_src mesh evaluated
    at the nodes of the level-L_dst mesh of the same patches (bilinear on
    every patch); returns a canonical vector of the destination mesh."""
    import torch
    u_fine = u_src
    nf, nc = 1 << L_src, 1 << L_dst
    U = _grid(u_fine, q, nf)                                   # [m, c, j, i]
    t = torch.arange(nc, dtype=torch.float64, device=u_fine.device) * ((nf - 1) / (nc - 1))
    i0 = torch.clamp(t.floor().long(), max=nf - 2)
    w = t - i0.double()
    i1 = i0 + 1
    # along i, then along j
    Ux = U[..., i0] * (1 - w) + U[..., i1] * w                 # [m, c, j, ic]
    Uxy = Ux[:, :, i0, :] * (1 - w)[:, None] + Ux[:, :, i1, :] * w[:, None]   # [m, c, jc, ic]
    return Uxy.permute(0, 2, 3, 1).reshape(-1).contiguous()


def level_record(make: Callable[[int], object], L: int, **solve_kw):
    """Assemble and solve one level; returns (record, canonical solution, K)."""
    import torch
    prob = make(L)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    K, f = qtt_assemble_stiffness(prob)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    u, info = qtt_solve(K, f, check=False, **solve_kw)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    r = u.ranks
    n = u.modes
    rec = {"d": L, "dofs": 2 * prob.q * 4 ** L, "ranks": r, "R_d": max(r),
           "N_d": sum(r[k] * n[k] * r[k + 1] for k in range(len(n))), "erank": info["erank"],
           "mem_K_mib": _bytes(K) / 2 ** 20, "mem_f_mib": _bytes(f) / 2 ** 20, "mem_u_mib": _bytes(u) / 2 ** 20,
           "assemble_s": t1 - t0, "solve_s": t2 - t1, "sweeps": info["sweeps"],
           "refinements": info["refinements"], "rel_residual": info["rel_residual"], "status": info["rc"]}
    return rec, qtt_to_full(u, ordering=QTT_ORDER_CANONICAL), K


def study(make: Callable[[int], object], levels: List[int], ref_level: int, tol: float = 1e-10,
          precision: int = QTT_MIXED, **solve_kw) -> List[Dict]:
    """Records for every level, with errors against the ref_level solution."""
    import torch

    def rel(e, ref, K):
        l2 = float(torch.linalg.norm(e) / torch.linalg.norm(ref))
        en = float(torch.sqrt(torch.clamp(torch.dot(e, qtt_fe_apply(K, e)), min=0.0)) /
                   torch.sqrt(torch.dot(ref, qtt_fe_apply(K, ref))))
        return l2, en

    ref_rec, u_ref, K_ref = level_record(make, ref_level, tol=tol, precision=precision, **solve_kw)
    q = make(ref_level).q
    out = []
    for L in levels:
        rec, u, K = level_record(make, L, tol=tol, precision=precision, **solve_kw)
        rec["err_l2"], rec["err_energy"] = rel(u_ref - interpolate(u, q, L, ref_level), u_ref, K_ref)
        ur = interpolate(u_ref, q, ref_level, L)
        rec["err_l2_nodal"], rec["err_energy_nodal"] = rel(u - ur, ur, K)
        out.append(rec)
    ref_rec["reference"] = True
    out.append(ref_rec)
    return out


def rates(records: List[Dict]) -> Dict[str, float]:
    """Least-squares rates over the records that carry errors: the algebraic
    orders p in err ~ h^p (h = 1 / (2^d - 1)) for L2 and energy, and the
    exponential rate b in err ~ exp(-b N_d)."""
    rs = [r for r in records if "err_l2" in r and r["err_l2"] > 0]
    if len(rs) < 2:
        return {}
    lh = np.log([1.0 / ((1 << r["d"]) - 1) for r in rs])
    out = {}
    for key in ("err_l2", "err_energy", "err_l2_nodal", "err_energy_nodal"):
        ly = np.log([r[key] for r in rs])
        out["order_" + key] = float(np.polyfit(lh, ly, 1)[0])
    nd = np.asarray([r["N_d"] for r in rs], dtype=float)
    out["exp_rate_err_energy_in_N_d"] = float(-np.polyfit(nd, np.log([r["err_energy"] for r in rs]), 1)[0])
    return out
