"""O-4: randomized rounding of the residual f - K u (oracle; test
infrastructure only -- imported by tests, never by the product path).

Randomize-then-orthogonalize TT rounding (Al Daas, Ballard, Cazeaux,
Hallman, Miedlar, Pasha, Reid and Saibaba, "Randomized algorithms for
rounding in the Tensor-Train format", SIAM J. Sci. Comput. 2023), applied to
y = f - K u written out as an explicit TT: the cores of K u by the MPO x MPS
product, then the block sum with f.  Plain NumPy in FP64, no structure of the
sum exploited:
  1. a Gaussian TT G with ranks l_b (l_0 = l_D = 1);
  2. right sketches W_D = [1], W_b = sum_i Y_b[:, i, :] W_{b+1} G_b[:, i, :]^T;
  3. left to right with M_0 = [1]: the (q_k n_k) x l_{k+1} matrix
     Z_k = (M_k Y_k) W_{k+1}; Q_k R = qr(Z_k); core k = Q_k;
     M_{k+1} = Q_k^T (M_k Y_k); the last core is M_{D-1} Y_{D-1}.
The result is the orthogonal projection of y onto the span of its
left-orthonormal factors.

Readings for parity with the engine: the sketch rank at bond b is
min(ell, R_b r_b + p_b, n_1 ... n_b, n_{b+1} ... n_D) (at least 1), i.e.
capped by the rank of the explicit sum and by the mode products; the
Gaussian entries come from the counter-based generator splitmix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
2014) and the Box-Muller transform: entry e (column-major) of core b uses the
counters 2e and 2e+1 under the key seed * 0x2545F4914F6CDD1D + b (mod 2^64).
"""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from . import tt

Cores = List[np.ndarray]

_M64 = (1 << 64) - 1


def mix64(z):
    """splitmix64 output function applied to z + golden gamma (uint64 arrays
    or Python ints)."""
    if isinstance(z, (int, np.integer)):
        z = (int(z) + 0x9E3779B97F4A7C15) & _M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def gaussian(key: int, count: int) -> np.ndarray:
    """count N(0, 1) samples: Box-Muller on two counter-based uniforms."""
    e = np.arange(count, dtype=np.uint64)
    k = np.uint64(key & _M64)
    with np.errstate(over="ignore"):
        a = mix64(k ^ mix64(np.uint64(2) * e))
        b = mix64(k ^ mix64(np.uint64(2) * e + np.uint64(1)))
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740993.0)   # (0, 1]
    u2 = (b >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)          # [0, 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def sketch_core(seed: int, b: int, shape: Sequence[int]) -> np.ndarray:
    key = (seed * 0x2545F4914F6CDD1D + b) & _M64
    return gaussian(key, int(np.prod(shape))).reshape(shape, order="F")


def residual_tt(K: Cores, u: Cores, f: Cores) -> Cores:
    """Explicit TT of f - K u (ranks p + R r)."""
    return tt.add(f, tt.scale(tt.matvec(K, u), -1.0))


def sketch_ranks(K: Cores, u: Cores, f: Cores, ell: int) -> List[int]:
    D = len(K)
    n = [c.shape[1] for c in K]
    lr = [1] * (D + 1)
    for b in range(1, D):
        rr = K[b].shape[0] * u[b].shape[0] + f[b].shape[0]
        left = math.prod(n[:b])
        right = math.prod(n[b:])
        lr[b] = max(1, min(ell, rr, left, right))
    return lr


def round_residual(K: Cores, u: Cores, f: Cores, ell: int, seed: int):
    """Rank-ell approximation of f - K u; returns (cores, norm of the result)."""
    y = residual_tt(K, u, f)
    D = len(y)
    lr = sketch_ranks(K, u, f, ell)
    G = [None] + [sketch_core(seed, b, (lr[b], y[b].shape[1], lr[b + 1])) for b in range(1, D)]
    W = [None] * (D + 1)
    W[D] = np.ones((1, 1))
    for b in range(D - 1, 0, -1):
        # W_b[s, l] = sum_{i, s', l'} Y_b[s, i, s'] W_{b+1}[s', l'] G_b[l, i, l']
        W[b] = np.einsum("sit,tm,lim->sl", y[b], W[b + 1], G[b], optimize=True)
    out = []
    M = np.ones((1, 1))
    for k in range(D):
        Y = np.einsum("qa,aib->qib", M, y[k])
        q, n, s = Y.shape
        if k == D - 1:
            out.append(Y)
            break
        Z = Y.reshape(q * n, s, order="F") @ W[k + 1]
        Q, _ = np.linalg.qr(Z, mode="reduced")
        out.append(Q.reshape(q, n, Q.shape[1], order="F"))
        M = Q.T @ Y.reshape(q * n, s, order="F")
    return out, float(np.linalg.norm(out[-1]))
