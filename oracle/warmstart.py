"""O-3: learned warm start (oracle; test infrastructure only).

A 3-layer MLP maps load/material parameters to fixed-rank QTT cores that seed
the AMEn sweeps.  Plain NumPy forward and backward (no autograd), written
from the definitions:

  features  phi = ((log10 E - 1.5) / 1.5, (nu - 0.325) / 0.125, cos theta, sin theta)
  layer 1   h1 = tanh(W1 phi + b1)            (width H)
  layer 2   h2 = tanh(W2 h1 + b2)             (width H)
  output    o  = W3 h2 + b3                    (P = sum of core sizes)
  cores     o is cut into rank-r cores (1,n1,r), (r,n2,r), ..., (r,nd,1),
            each stored column-major; the predicted solution is
            u_hat = (amp / E) * TT(o)  (the scale folded into core 1).

Loss (gauge invariant, per sample, normalised by the target):
  l = ||X_hat - X||^2 / ||X||^2 = (<X_hat,X_hat> - 2 <X_hat,X> + <X,X>) / <X,X>
with X = (E / amp) u the method's solution divided by the same scale and
X_hat = TT(o).  Inner products use left transfer matrices; the gradient with
respect to core k is 2 (Lhh_k X_hat_k Rhh_k - Lhx_k X_k Rhx_k) / <X,X>, with
left/right environments L, R of the two inner products.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np


def features(params: np.ndarray) -> np.ndarray:
    """params rows (E, nu, amp, theta) -> (B, 4) features."""
    E, nu, amp, th = params[:, 0], params[:, 1], params[:, 2], params[:, 3]
    return np.stack([(np.log10(E) - 1.5) / 1.5, (nu - 0.325) / 0.125, np.cos(th), np.sin(th)], axis=1)


def core_shapes(modes: Sequence[int], r: int) -> List[Tuple[int, int, int]]:
    d = len(modes)
    out = []
    for k, n in enumerate(modes):
        out.append((1 if k == 0 else r, n, 1 if k == d - 1 else r))
    return out


def n_outputs(modes: Sequence[int], r: int) -> int:
    return int(sum(a * b * c for a, b, c in core_shapes(modes, r)))


def init_params(seed: int, n_in: int, H: int, P: int, out_scale: float = 0.05):
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, n_in)) / math.sqrt(n_in)
    W2 = rng.standard_normal((H, H)) / math.sqrt(H)
    W3 = rng.standard_normal((P, H)) * (out_scale / math.sqrt(H))
    return {"W1": W1, "b1": np.zeros(H), "W2": W2, "b2": np.zeros(H), "W3": W3, "b3": np.zeros(P)}


def forward(p, phi: np.ndarray):
    """phi (B, n_in) -> (o (B, P), cache)."""
    a1 = phi @ p["W1"].T + p["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(a2)
    o = h2 @ p["W3"].T + p["b3"]
    return o, (phi, h1, h2)


def backward(p, cache, go: np.ndarray):
    """Gradients of the parameters given dL/do (B, P)."""
    phi, h1, h2 = cache
    g = {}
    g["W3"] = go.T @ h2
    g["b3"] = go.sum(axis=0)
    gh2 = go @ p["W3"]
    ga2 = gh2 * (1.0 - h2 * h2)
    g["W2"] = ga2.T @ h1
    g["b2"] = ga2.sum(axis=0)
    gh1 = ga2 @ p["W2"]
    ga1 = gh1 * (1.0 - h1 * h1)
    g["W1"] = ga1.T @ phi
    g["b1"] = ga1.sum(axis=0)
    return g


def split_cores(o_row: np.ndarray, modes: Sequence[int], r: int) -> List[np.ndarray]:
    """Cut one output row into column-major cores."""
    cores, off = [], 0
    for (a, n, b) in core_shapes(modes, r):
        sz = a * n * b
        cores.append(o_row[off:off + sz].reshape((a, n, b), order="F"))
        off += sz
    return cores


def _inner_envs(X: List[np.ndarray], Y: List[np.ndarray]):
    """Left environments L[k] (before core k) and right R[k] (after core k)
    of <X, Y>."""
    d = len(X)
    L = [np.ones((1, 1))]
    for k in range(d):
        L.append(np.einsum("ab,aic,bid->cd", L[-1], X[k], Y[k]))
    R = [None] * (d + 1)
    R[d] = np.ones((1, 1))
    for k in range(d - 1, -1, -1):
        R[k] = np.einsum("aic,bid,cd->ab", X[k], Y[k], R[k + 1])
    return L, R


def tt_loss_and_grad(Xh: List[np.ndarray], X: List[np.ndarray]):
    """l = ||Xh - X||^2 / ||X||^2 and dl/dXh (list of cores)."""
    Lhh, Rhh = _inner_envs(Xh, Xh)
    Lhx, Rhx = _inner_envs(Xh, X)
    Lxx, _ = _inner_envs(X, X)
    hh = float(Lhh[-1][0, 0])
    hx = float(Lhx[-1][0, 0])
    xx = float(Lxx[-1][0, 0])
    loss = (hh - 2.0 * hx + xx) / xx
    grads = []
    for k in range(len(Xh)):
        g_hh = np.einsum("ab,bid,cd->aic", Lhh[k], Xh[k], Rhh[k + 1])
        g_hx = np.einsum("ab,bid,cd->aic", Lhx[k], X[k], Rhx[k + 1])
        grads.append(2.0 * (g_hh - g_hx) / xx)
    return loss, grads


def batch_loss_and_grad(o: np.ndarray, targets: Sequence[List[np.ndarray]], modes, r: int):
    """Mean loss over the batch and dL/do (B, P)."""
    B = o.shape[0]
    go = np.zeros_like(o)
    tot = 0.0
    for b in range(B):
        cores = split_cores(o[b], modes, r)
        l, gc = tt_loss_and_grad(cores, targets[b])
        tot += l
        go[b] = np.concatenate([g.reshape(-1, order="F") for g in gc]) / B
    return tot / B, go


def adam_step(p, g, state, lr: float, t: int, b1=0.9, b2=0.999, eps=1e-8):
    for k in p:
        m = state.setdefault("m" + k, np.zeros_like(p[k]))
        v = state.setdefault("v" + k, np.zeros_like(p[k]))
        m[:] = b1 * m + (1 - b1) * g[k]
        v[:] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)
