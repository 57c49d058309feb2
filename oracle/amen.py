"""O-2: AMEn solver for A x = y in TT format (oracle; test infrastructure).

The paper solves K u = f "with the AMEn solver" (Sections 3, 3.7 and 5.1)
and cites Dolgov & Savostyanov (2014) without restating it.  This module is
a plain restatement of one-site AMEn with residual-based enrichment written
from that method's mathematics, in the reading fixed for this project:

  0. inputs: operator A (MPO), right-hand side y (MPS), initial guess x0,
     initial residual proxy z0 (random, rank rho), tolerance eps;
  1. right-orthogonalise x and z, build all right interfaces;
  2. sweep k = 1..D (left to right):
       a. local system B_k = Phi_L(x,A,x) x A_k x Phi_R(x,A,x), local rhs
          g_k = Psi_L(x,y) y_k Psi_R(x,y);
       b. local residual of the current core ||B_k x_k - g_k|| / ||g_k||;
          its maximum over k is the sweep's convergence measure;
       c. solve B_k x_k = g_k (dense LU up to `local_direct_max` unknowns,
          otherwise restarted GMRES warm-started from x_k);
       d. k < D: truncated SVD of the left unfolding x_k = U S V^T keeping
          the smallest rank whose truncated core has local residual <=
          eps / sqrt(D) (relative to ||g_k||), found by bisection;
       e. residual-proxy core: z_k = orth of the local residual projected on
          z's left and right interfaces; enrichment block = the residual
          projected on x's left and z's right interfaces;
       f. U <- orth([U, enrichment]); the next core absorbs R [S V^T; 0];
       g. update the left interfaces of x and z;
  3. stop when the sweep's maximum local residual is <= eps; otherwise
     restart at step 1 (one-directional sweeps).
Interfaces use the index convention Phi[test, operator, trial].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse.linalg as spla

from . import tt

Cores = List[np.ndarray]


@dataclass
class AmenInfo:
    sweeps: int = 0
    max_res_history: List[float] = field(default_factory=list)
    ranks: List[int] = field(default_factory=list)
    converged: bool = False
    local_iters: int = 0


def _left_XAX(Phi, X, Ak, Y):
    """Phi'[b, B, d] = sum Phi[a, A, c] X[a, i, b] A[A, i, j, B] Y[c, j, d]."""
    t = np.tensordot(Phi, X, axes=([0], [0]))               # [A, c, i, b]
    t = np.tensordot(t, Ak, axes=([0, 2], [0, 1]))          # [c, b, j, B]
    t = np.tensordot(t, Y, axes=([0, 2], [0, 1]))           # [b, B, d]
    return t


def _right_XAX(Phi, X, Ak, Y):
    """Phi[a, A, c] = sum X[a, i, b] A[A, i, j, B] Y[c, j, d] Phi'[b, B, d]."""
    t = np.tensordot(Y, Phi, axes=([2], [2]))               # [c, j, b, B]
    t = np.tensordot(t, Ak, axes=([1, 3], [2, 3]))          # [c, b, A, i]
    t = np.tensordot(X, t, axes=([1, 2], [3, 1]))           # [a, c, A]
    return t.transpose(0, 2, 1)


def _left_XY(Psi, X, Yk):
    """Psi'[b, d] = sum Psi[a, c] X[a, i, b] y[c, i, d]."""
    return np.einsum("ac,aib,cid->bd", Psi, X, Yk, optimize=True)


def _right_XY(Psi, X, Yk):
    """Psi[a, c] = sum X[a, i, b] y[c, i, d] Psi'[b, d]."""
    return np.einsum("aib,cid,bd->ac", X, Yk, Psi, optimize=True)


def local_apply(PhiL, Ak, PhiR, x):
    """(B x)[a, i, b] = sum PhiL[a, A, a'] A[A, i, j, B] PhiR[b, B, b'] x[a', j, b'],
    contracted in three steps: over b', then over (j, B), then over (a', A)."""
    t1 = np.tensordot(x, PhiR, axes=([2], [2]))            # [a', j, b, B]
    t2 = np.tensordot(t1, Ak, axes=([1, 3], [2, 3]))       # [a', b, A, i]
    y = np.tensordot(PhiL, t2, axes=([1, 2], [2, 0]))      # [a, b, i]
    return y.transpose(0, 2, 1)


def local_rhs(PsiL, yk, PsiR):
    """g[a, i, b] = sum PsiL[a, c] y[c, i, d] PsiR[b, d]."""
    t = np.tensordot(PsiL, yk, axes=([1], [0]))             # [a, i, d]
    return np.tensordot(t, PsiR, axes=([2], [1]))           # [a, i, b]


def local_matrix(PhiL, Ak, PhiR):
    """Dense B with column-major flattening of (a, i, b) for rows and
    (a', j, b') for columns."""
    r0 = PhiL.shape[0]
    r1 = PhiR.shape[0]
    n = Ak.shape[1]
    t = np.tensordot(PhiL, Ak, axes=([1], [0]))             # [a, a', i, j, B]
    B = np.tensordot(t, PhiR, axes=([4], [1]))              # [a, a', i, j, b, b']
    N = r0 * n * r1
    # rows (a, i, b) and columns (a', j, b'), first index fastest
    return B.transpose(4, 2, 0, 5, 3, 1).reshape(N, N)


def _vec(x):
    return x.reshape(-1, order="F")


def _unvec(v, shape):
    return v.reshape(shape, order="F")


def _orth_right(cores: Cores) -> Cores:
    return tt.right_orthogonalize([c.copy() for c in cores])


def amen_solve(A: Cores, y: Cores, x0: Cores, z0: Cores, eps: float,
               max_sweeps: int = 20, max_rank: int = 1 << 30,
               local_direct_max: int = 2500, gmres_restart: int = 40,
               gmres_maxiter: int = 4, verbose: bool = False, on_sweep=None):
    """Solve A x = y; returns (x cores, AmenInfo).  on_sweep(sweep, max_res),
    if given, is called after every sweep (timing instrumentation only)."""
    D = len(A)
    x = [c.copy() for c in x0]
    z = [c.copy() for c in z0]
    info = AmenInfo()
    delta = eps / math.sqrt(D)
    for sweep in range(max_sweeps):
        x = _orth_right(x)
        z = _orth_right(z)
        one = np.ones((1, 1, 1))
        XAX_R = [None] * (D + 1)
        XY_R = [None] * (D + 1)
        ZAX_R = [None] * (D + 1)
        ZY_R = [None] * (D + 1)
        XAX_R[D] = one
        XY_R[D] = np.ones((1, 1))
        ZAX_R[D] = one
        ZY_R[D] = np.ones((1, 1))
        for k in range(D - 1, 0, -1):
            XAX_R[k] = _right_XAX(XAX_R[k + 1], x[k], A[k], x[k])
            XY_R[k] = _right_XY(XY_R[k + 1], x[k], y[k])
            ZAX_R[k] = _right_XAX(ZAX_R[k + 1], z[k], A[k], x[k])
            ZY_R[k] = _right_XY(ZY_R[k + 1], z[k], y[k])
        XAX_L = one
        XY_L = np.ones((1, 1))
        ZAX_L = one
        ZY_L = np.ones((1, 1))
        max_res = 0.0
        for k in range(D):
            PhiR = XAX_R[k + 1]
            PsiR = XY_R[k + 1]
            g = local_rhs(XY_L, y[k], PsiR)
            gn = np.linalg.norm(g)
            xk = x[k]
            res = np.linalg.norm(local_apply(XAX_L, A[k], PhiR, xk) - g) / (gn if gn > 0 else 1.0)
            max_res = max(max_res, res)
            shape = xk.shape
            N = xk.size
            if N <= local_direct_max:
                B = local_matrix(XAX_L, A[k], PhiR)
                sol = np.linalg.solve(B, _vec(g))
            else:
                op = spla.LinearOperator((N, N), matvec=lambda v: _vec(local_apply(XAX_L, A[k], PhiR, _unvec(v, shape))),
                                         dtype=np.float64)
                sol, _ = spla.gmres(op, _vec(g), x0=_vec(xk), rtol=delta, restart=gmres_restart,
                                    maxiter=gmres_maxiter, atol=0.0)
                info.local_iters += 1
            xk = _unvec(sol, shape)
            if k == D - 1:
                x[k] = xk
                break
            r0, n, r1 = shape
            U, s, Vt = np.linalg.svd(xk.reshape(r0 * n, r1, order="F"), full_matrices=False)
            # residual-norm truncation: the smallest rank whose truncated core
            # keeps the local residual within delta (or within twice what the
            # local solve itself reached, if that is larger)
            res_sol = np.linalg.norm(local_apply(XAX_L, A[k], PhiR, xk) - g) / (gn if gn > 0 else 1.0)
            thr = max(delta, 2.0 * res_sol) * (gn if gn > 0 else 1.0)
            rk = len(s)
            lo = 1
            while lo < rk:
                mid = (lo + rk) // 2
                cand = ((U[:, :mid] * s[:mid]) @ Vt[:mid]).reshape(shape, order="F")
                if np.linalg.norm(local_apply(XAX_L, A[k], PhiR, cand) - g) <= thr:
                    rk = mid
                else:
                    lo = mid + 1
            rk = min(rk, max_rank)
            U, s, Vt = U[:, :rk], s[:rk], Vt[:rk]
            xt = (U * s) @ Vt                                    # truncated core, (r0 n) x r1
            xt3 = xt.reshape(r0, n, r1, order="F")
            # residual projected on z's left / right interfaces -> new z core
            zres = local_rhs(ZY_L, y[k], ZY_R[k + 1]) - local_apply(ZAX_L, A[k], ZAX_R[k + 1], xt3)
            rz0, _, rz1 = zres.shape
            Qz, _ = np.linalg.qr(zres.reshape(rz0 * n, rz1, order="F"))
            zk = Qz.reshape(rz0, n, Qz.shape[1], order="F")
            # enrichment: residual on x's left and z's right interfaces
            enr = local_rhs(XY_L, y[k], ZY_R[k + 1]) - local_apply(XAX_L, A[k], ZAX_R[k + 1], xt3)
            Uaug = np.concatenate([U, enr.reshape(r0 * n, -1, order="F")], axis=1)
            Q, R = np.linalg.qr(Uaug)
            newr = Q.shape[1]
            SV = np.zeros((Uaug.shape[1], r1))
            SV[:rk] = s[:, None] * Vt
            carry = R @ SV                                       # newr x r1
            x[k] = Q.reshape(r0, n, newr, order="F")
            x[k + 1] = np.einsum("ab,bnc->anc", carry, x[k + 1])
            # z: the next core is re-expressed in the new z basis only through
            # the interfaces; z[k+1] keeps its right-orthogonal content
            if zk.shape[2] != z[k].shape[2]:
                # rank of z cannot exceed (rz0 n); keep the next core consistent
                z[k + 1] = z[k + 1][: zk.shape[2]]
            z[k] = zk
            XAX_L = _left_XAX(XAX_L, x[k], A[k], x[k])
            XY_L = _left_XY(XY_L, x[k], y[k])
            ZAX_L = _left_XAX(ZAX_L, z[k], A[k], x[k])
            ZY_L = _left_XY(ZY_L, z[k], y[k])
        info.sweeps = sweep + 1
        info.max_res_history.append(max_res)
        if on_sweep is not None:
            on_sweep(sweep + 1, max_res)
        if verbose:
            print(f"sweep {sweep + 1}: max local res {max_res:.3e} ranks {tt.ranks(x)}")
        if max_res <= eps:
            info.converged = True
            break
    info.ranks = tt.ranks(x)
    return x, info
