"""Learned warm start for the plate family: a 3-layer MLP from
(E, nu, traction amplitude, angle) to rank-r QTT cores that seed qtt_solve.

Weights live in PyTorch device tensors (memory only); the forward pass, the
backward pass, the gauge-invariant TT loss and the Adam update run in the
library's kernels (qtt_ws_*).  The network predicts the solution scaled by
E / amp, and the warm start is (amp / E) times the predicted tensor: the
plane-stress solution is linear in the traction and in 1 / E.

Training targets are method-generated: for every nu of a grid the engine
solves the two unit-traction problems (x and y traction, E = 1), and each
training sample's target is the superposition cos(theta) U_x(nu) +
sin(theta) U_y(nu), passed to the loss as coefficients over those basis
solutions (the loss never forms the sum).
"""
from __future__ import annotations

import ctypes as C
import math
from typing import List, Sequence

import numpy as np

from . import QTT, QTT_F32, _check, _stream, lib, qtt_assemble_stiffness, qtt_solve


def features(params: np.ndarray) -> np.ndarray:
    """(B, 4) rows (E, nu, amp, theta) -> (4, B) float32, column-major batch."""
    E, nu, amp, th = params[:, 0], params[:, 1], params[:, 2], params[:, 3]
    f = np.stack([(np.log10(E) - 1.5) / 1.5, (nu - 0.325) / 0.125, np.cos(th), np.sin(th)], axis=0)
    return np.ascontiguousarray(f.T.astype(np.float32))          # (B, 4) rows == (4 x B) column-major


def n_outputs(modes: Sequence[int], r: int) -> int:
    d = len(modes)
    return sum((1 if k == 0 else r) * n * (1 if k == d - 1 else r) for k, n in enumerate(modes))


def _p(t):
    return C.c_void_p(t.data_ptr())


class WarmStartMLP:
    """4 -> H -> H -> P MLP (tanh) predicting rank-r cores for `modes`."""

    def __init__(self, modes: Sequence[int], r: int = 16, H: int = 256, seed: int = 0, out_scale: float = 0.25):
        import torch
        self.modes = list(modes)
        self.r = r
        self.H = H
        self.nin = 4
        self.P = n_outputs(modes, r)
        g = torch.Generator().manual_seed(seed)
        dev = "cuda"
        # a column-major (rows x cols) matrix is a contiguous torch tensor of
        # shape (cols, rows): W1 is H x nin, W2 H x H, W3 P x H
        self.params = {
            "W1": (torch.randn(self.nin, H, generator=g) / math.sqrt(self.nin)).to(dev),
            "b1": torch.zeros(H, device=dev),
            "W2": (torch.randn(H, H, generator=g) / math.sqrt(H)).to(dev),
            "b2": torch.zeros(H, device=dev),
            "W3": (torch.randn(H, self.P, generator=g) * (out_scale / math.sqrt(H))).to(dev),
            "b3": torch.zeros(self.P, device=dev),
        }
        # targets are learned divided by this norm scale (set by train), so
        # that the predicted TT starts at a norm comparable to the targets':
        # with a scale far off, a product of D cores and its gradients vanish
        self.target_scale = 1.0
        self.m = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.t = 0

    # -- kernels ---------------------------------------------------------------
    def forward(self, phi, stream=None):
        """phi: torch (B, 4) float32 on cuda -> (out (B, P), h1, h2)."""
        import torch
        B = phi.shape[0]
        h1 = torch.empty(B, self.H, device="cuda")
        h2 = torch.empty(B, self.H, device="cuda")
        out = torch.empty(B, self.P, device="cuda")
        p = self.params
        _check(lib().qtt_ws_forward(B, self.nin, self.H, self.P, _p(p["W1"]), _p(p["b1"]), _p(p["W2"]), _p(p["b2"]),
                                    _p(p["W3"]), _p(p["b3"]), _p(phi), _p(h1), _p(h2), _p(out), _stream(stream)),
               "qtt_ws_forward")
        return out, h1, h2

    def basis_gram(self, basis: List[QTT], stream=None) -> np.ndarray:
        n = len(basis)
        arr = (C.c_void_p * n)(*[b.handle for b in basis])
        g = np.zeros((n, n))
        _check(lib().qtt_ws_basis_gram(len(self.modes), n, arr, g.ctypes.data_as(C.POINTER(C.c_double)),
                                       _stream(stream)), "qtt_ws_basis_gram")
        return g

    def loss_and_grad(self, out, basis: List[QTT], coef: np.ndarray, gram: np.ndarray = None, stream=None):
        import torch
        B = out.shape[0]
        loss = torch.empty(B, device="cuda")
        gout = torch.empty_like(out)
        arr = (C.c_void_p * len(basis))(*[b.handle for b in basis])
        modes = (C.c_int * len(self.modes))(*self.modes)
        cf = np.ascontiguousarray(coef, dtype=np.float64)
        gp = None
        if gram is not None:
            gram = np.ascontiguousarray(gram, dtype=np.float64)
            gp = gram.ctypes.data_as(C.POINTER(C.c_double))
        _check(lib().qtt_ws_tt_loss(B, len(self.modes), modes, self.r, _p(out), len(basis), arr,
                                    cf.ctypes.data_as(C.POINTER(C.c_double)), gp, _p(loss), _p(gout),
                                    _stream(stream)), "qtt_ws_tt_loss")
        return loss, gout

    def backward(self, phi, h1, h2, gout, stream=None):
        import torch
        B = phi.shape[0]
        g = {k: torch.empty_like(v) for k, v in self.params.items()}
        work = torch.empty(2 * self.H * B, device="cuda")
        p = self.params
        _check(lib().qtt_ws_backward(B, self.nin, self.H, self.P, _p(p["W2"]), _p(p["W3"]), _p(phi), _p(h1), _p(h2),
                                     _p(gout), _p(g["W1"]), _p(g["b1"]), _p(g["W2"]), _p(g["b2"]), _p(g["W3"]),
                                     _p(g["b3"]), _p(work), _stream(stream)), "qtt_ws_backward")
        return g

    def adam(self, g, lr=1e-3, stream=None):
        self.t += 1
        for k, w in self.params.items():
            _check(lib().qtt_ws_adam(w.numel(), _p(w), _p(g[k]), _p(self.m[k]), _p(self.v[k]), lr, 0.9, 0.999, 1e-8,
                                     self.t, _stream(stream)), "qtt_ws_adam")

    def train_step(self, params: np.ndarray, basis: List[QTT], coef: np.ndarray, lr=1e-3, gram=None):
        import torch
        phi = torch.from_numpy(features(params)).cuda()
        out, h1, h2 = self.forward(phi)
        loss, gout = self.loss_and_grad(out, basis, coef, gram)
        g = self.backward(phi, h1, h2, gout)
        self.adam(g, lr)
        return float(loss.mean())

    def predict(self, params: np.ndarray) -> List[QTT]:
        """Warm starts (amp / E) * TT(out) for each parameter row."""
        import torch
        phi = torch.from_numpy(features(params)).cuda()
        out, _, _ = self.forward(phi)
        xs = []
        modes = (C.c_int * len(self.modes))(*self.modes)
        for b in range(params.shape[0]):
            h = C.c_void_p()
            scale = float(params[b, 2] / params[b, 0]) * self.target_scale
            _check(lib().qtt_ws_to_tensor(C.c_void_p(out[b].data_ptr()), len(self.modes), modes, self.r, scale,
                                          C.byref(h), _stream(None)), "qtt_ws_to_tensor")
            xs.append(QTT(h))
        return xs


def basis_solutions(L: int, nus: Sequence[float], tol: float = 1e-8, **solve_kw):
    """Unit-traction solutions U_x(nu), U_y(nu) at E = 1 for every nu; returns
    a list [U_x(nu_0), U_y(nu_0), U_x(nu_1), ...] of FP64 QTT tensors."""
    import workloads as W
    from . import qtt_solve_batched
    probs = [W.plate_top_traction(L, 1.0, float(nu), 1.0, th) for nu in nus for th in (0.0, math.pi / 2)]
    KF = [qtt_assemble_stiffness(p) for p in probs]
    us, infos = qtt_solve_batched([k for k, _ in KF], [f for _, f in KF], tol=tol, **solve_kw)
    return us


def dataset(seed: int, count: int, nus: Sequence[float]):
    """Training parameters on the nu grid and the superposition coefficients
    of their scaled targets over basis_solutions(nus)."""
    import workloads as W
    P = W.plate_params(seed, count)
    rng = np.random.default_rng(seed + 1000)
    idx = rng.integers(0, len(nus), count)
    P[:, 1] = np.asarray(nus)[idx]
    coef = np.zeros((count, 2 * len(nus)))
    coef[np.arange(count), 2 * idx] = np.cos(P[:, 3])
    coef[np.arange(count), 2 * idx + 1] = np.sin(P[:, 3])
    return P, coef


def train(net: WarmStartMLP, basis: List[QTT], P: np.ndarray, coef: np.ndarray, steps: int = 300, batch: int = 32,
          lr: float = 2e-3, seed: int = 0):
    """Adam on random mini-batches; the learning rate decays by 10x over the
    run.  Targets are divided by the RMS norm of the basis solutions (the
    network's target_scale).  Returns the per-step mean (relative) losses."""
    gram = net.basis_gram(basis)
    net.target_scale = float(np.sqrt(np.mean(np.diag(gram))))
    coef = np.asarray(coef) / net.target_scale
    rng = np.random.default_rng(seed)
    losses = []
    for st in range(steps):
        idx = rng.integers(0, len(P), batch)
        a = lr * (0.1 ** (st / max(1, steps - 1)))
        losses.append(net.train_step(P[idx], basis, coef[idx], lr=a, gram=gram))
    return losses


class SuperpositionStart:
    """Non-learned warm start for the plate family: the plane-stress
    solution is linear in the traction and in 1/E, and smooth in nu, so
    stored method solutions of the two unit tractions on a nu grid give

        x0 = (amp / E) * sum_j w_j(nu) (cos(theta) U_x(nu_j) + sin(theta) U_y(nu_j)),

    with w_j the Lagrange weights of the `order` grid points nearest to nu
    (exact at grid points).  The sum is formed and rounded by the library's
    qtt_axpby / qtt_round.  Its residual is of the size of the interpolation
    error in nu (a smooth field), unlike a rank-limited learned start whose
    error reaches the high frequencies that K amplifies."""

    def __init__(self, L: int, nus: Sequence[float], order: int = 3, tol: float = 1e-8, round_tol: float = 1e-9,
                 **solve_kw):
        self.nus = np.asarray(sorted(nus), dtype=float)
        self.order = max(1, min(order, len(self.nus)))
        self.round_tol = round_tol
        self.basis = basis_solutions(L, list(self.nus), tol=tol, **solve_kw)   # U_x(nu_0), U_y(nu_0), ...

    def weights(self, nu: float):
        """Indices and Lagrange weights of the nearest `order` grid points."""
        idx = np.argsort(np.abs(self.nus - nu))[:self.order]
        idx = np.sort(idx)
        xs = self.nus[idx]
        w = []
        for a, xa in enumerate(xs):
            p = 1.0
            for b, xb in enumerate(xs):
                if b != a:
                    p *= (nu - xb) / (xa - xb)
            w.append(p)
        return idx, np.asarray(w)

    def predict(self, params: np.ndarray) -> List[QTT]:
        from . import qtt_axpby, qtt_round
        out = []
        for E, nu, amp, th in params:
            idx, w = self.weights(float(nu))
            x = None
            for j, wj in zip(idx, w):
                cx, cy = float(wj * math.cos(th) * amp / E), float(wj * math.sin(th) * amp / E)
                term = qtt_axpby(cx, self.basis[2 * j], cy, self.basis[2 * j + 1])
                x = term if x is None else qtt_axpby(1.0, x, 1.0, term)
                qtt_round(x, self.round_tol)
            out.append(x)
        return out
