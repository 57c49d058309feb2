"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds problem *descriptions* and random numbers only: patch
layouts, material constants, boundary flags, load coefficients, and random
TT cores / initial guesses drawn from seeded generators.  It contains none of
the method's arithmetic (no FE integrals, no TT algebra), so both sides of a
parity test can take their inputs from here without sharing any computation.

Geometry follows the domain partitioning of Section 3.1: the domain is a
union of q unit-square patches, each placed at an integer offset (ox, oy).
Every patch carries n = 2^L nodes per side (Section 3.2), so the mesh spacing
is h = 1/(n-1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

# Boundary flags per patch side, Section 3.8 (clamped / rollers).
FIX_X = 1          # u_x = 0 on the side (roller)
FIX_Y = 2          # u_y = 0 on the side (roller)
CLAMP = FIX_X | FIX_Y

# Side numbering used in `bc` and `traction` entries.
LEFT, RIGHT, BOTTOM, TOP = 0, 1, 2, 3

# 1D factor kinds of a separable body-force term f_c(x, y) = a * g(x) * h(y);
# x and y are global coordinates: 1, t, sin(pi t), cos(pi t), t^2.
ONE, LIN, SINPI, COSPI, QUAD = 0, 1, 2, 3, 4


@dataclasses.dataclass
class Problem:
    """Plane-stress elasticity problem on q unit-square patches.

    Attributes
    ----------
    L        : levels; n = 2^L nodes per patch side.
    patches  : list of integer offsets (ox, oy), one per patch.
    E, nu    : Young's modulus and Poisson ratio (plane stress).
    bc       : per patch, four side flags (LEFT, RIGHT, BOTTOM, TOP), each an
               OR of FIX_X / FIX_Y.
    body     : separable body-force terms (component, coeff, xkind, ykind).
    traction : constant edge tractions (patch, side, tx, ty).
    gamma    : concatenation penalty; 0 selects the mean diagonal of K_xx.
    dirichlet: prescribed displacement u0 on the constrained sides, as
               separable terms (component, coeff, xkind, ykind) of u0_c(x, y)
               in global coordinates (empty: homogeneous conditions).
    """

    L: int
    patches: List[Tuple[int, int]]
    E: float
    nu: float
    bc: List[Tuple[int, int, int, int]]
    body: List[Tuple[int, float, int, int]] = dataclasses.field(default_factory=list)
    traction: List[Tuple[int, int, float, float]] = dataclasses.field(default_factory=list)
    gamma: float = 0.0
    dirichlet: List[Tuple[int, float, int, int]] = dataclasses.field(default_factory=list)

    @property
    def q(self) -> int:
        return len(self.patches)

    @property
    def n(self) -> int:
        return 1 << self.L

    @property
    def ndof(self) -> int:
        return 2 * self.q * (1 << (2 * self.L))


# ----------------------------------------------------------------------------
# Named workloads (shapes of the paper's experiments, Section 5)
# ----------------------------------------------------------------------------

def plate_body_force(L: int, E: float = 1.0, nu: float = 0.3) -> Problem:
    """Unit-square plate, left edge clamped, uniform body force (0, -1)."""
    return Problem(L=L, patches=[(0, 0)], E=E, nu=nu,
                   bc=[(CLAMP, 0, 0, 0)],
                   body=[(1, -1.0, ONE, ONE)])


def plate_traction_smooth(L: int, E: float = 1.0, nu: float = 0.3) -> Problem:
    """Plate clamped on the left, traction (1, 0) on the right edge and body
    force (sin(pi x) sin(pi y), x y)."""
    return Problem(L=L, patches=[(0, 0)], E=E, nu=nu,
                   bc=[(CLAMP, 0, 0, 0)],
                   body=[(0, 1.0, SINPI, SINPI), (1, 1.0, LIN, LIN)],
                   traction=[(0, RIGHT, 1.0, 0.0)])


def lshape_shear(L: int, E: float = 210.0, nu: float = 0.3) -> Problem:
    """L-shaped panel of three unit squares [0,1]^2, [1,2]x[0,1], [0,1]x[1,2];
    clamped on y = 0, unit shear traction (1, 0) on the top edges."""
    return Problem(L=L, patches=[(0, 0), (1, 0), (0, 1)], E=E, nu=nu,
                   bc=[(0, 0, CLAMP, 0), (0, 0, CLAMP, 0), (0, 0, 0, 0)],
                   traction=[(1, TOP, 1.0, 0.0), (2, TOP, 1.0, 0.0)])


def two_patch_strip(L: int, E: float = 1.0, nu: float = 0.3) -> Problem:
    """Two side-by-side unit squares, left end clamped, top-edge traction."""
    return Problem(L=L, patches=[(0, 0), (1, 0)], E=E, nu=nu,
                   bc=[(CLAMP, 0, 0, 0), (0, 0, 0, 0)],
                   traction=[(0, TOP, 0.0, -1.0), (1, TOP, 0.0, -1.0)])


def plate_top_traction(L: int, E: float, nu: float, amp: float, theta: float) -> Problem:
    """Plate clamped on the left with a constant traction of amplitude `amp`
    at angle `theta` on the top edge (the parameter family of the learned
    warm start)."""
    return Problem(L=L, patches=[(0, 0)], E=E, nu=nu,
                   bc=[(CLAMP, 0, 0, 0)],
                   traction=[(0, TOP, amp * math.cos(theta), amp * math.sin(theta))])


def patch_test(L: int, patches=((0, 0),), E: float = 5.0, nu: float = 0.3) -> Problem:
    """Patch test: every outer side clamped to the linear field
    u0 = (0.1 + 0.2 x - 0.3 y, -0.05 + 0.1 x + 0.25 y), no loads, so the
    finite-element solution is u0 itself at every node."""
    ps = list(patches)
    occupied = set(ps)
    bc = []
    for (ox, oy) in ps:
        nb = [(ox - 1, oy), (ox + 1, oy), (ox, oy - 1), (ox, oy + 1)]
        bc.append(tuple(0 if q in occupied else CLAMP for q in nb))
    u0 = [(0, 0.1, ONE, ONE), (0, 0.2, LIN, ONE), (0, -0.3, ONE, LIN),
          (1, -0.05, ONE, ONE), (1, 0.1, LIN, ONE), (1, 0.25, ONE, LIN)]
    return Problem(L=L, patches=ps, E=E, nu=nu, bc=bc, dirichlet=u0)


def plate_prescribed_edge(L: int, E: float = 2.0, nu: float = 0.3) -> Problem:
    """Plate clamped on the left with the right edge pulled to the
    prescribed displacement u0 = (0.01 (1 + y), 0.02 sin(pi y)); top edge
    traction (0, -0.5)."""
    return Problem(L=L, patches=[(0, 0)], E=E, nu=nu, bc=[(CLAMP, CLAMP, 0, 0)],
                   traction=[(0, TOP, 0.0, -0.5)],
                   dirichlet=[(0, 0.01, ONE, ONE), (0, 0.01, ONE, LIN), (1, 0.02, ONE, SINPI)])


def plate_manufactured(L: int, E: float = 1.0, nu: float = 0.3) -> Problem:
    """Fully clamped plate whose exact plane-stress solution is
    u = (sin(pi x) sin(pi y), 0): the body force -div sigma(u) is
    f_x = e pi^2 (3 - nu) / 2 sin(pi x) sin(pi y),
    f_y = -e pi^2 (1 + nu) / 2 cos(pi x) cos(pi y), e = E / (1 - nu^2).
    A smooth solution without corner singularities (the Q1 orders hold)."""
    e = E / (1.0 - nu * nu)
    return Problem(L=L, patches=[(0, 0)], E=E, nu=nu, bc=[(CLAMP, CLAMP, CLAMP, CLAMP)],
                   body=[(0, e * math.pi ** 2 * (3.0 - nu) / 2.0, SINPI, SINPI),
                         (1, -e * math.pi ** 2 * (1.0 + nu) / 2.0, COSPI, COSPI)])


def plate_params(seed: int, count: int) -> np.ndarray:
    """(E, nu, amp, theta) rows: E log-uniform in [1, 1000], nu ~ U(0.2, 0.45),
    amp ~ U(0.5, 2), theta ~ U(0, 2 pi)."""
    rng = np.random.default_rng(seed)
    E = 10.0 ** rng.uniform(0.0, 3.0, count)
    nu = rng.uniform(0.2, 0.45, count)
    amp = rng.uniform(0.5, 2.0, count)
    theta = rng.uniform(0.0, 2.0 * math.pi, count)
    return np.stack([E, nu, amp, theta], axis=1)


def mixed_batch(seed: int, count: int, levels: Sequence[int] = (8, 9, 10, 11, 12, 13)) -> List[Problem]:
    """Uneven batch: q in {1, 2, 3}, L uniform over `levels`, material and
    top-edge traction drawn as in `plate_params`."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        q = int(rng.integers(1, 4))
        L = int(rng.choice(np.asarray(levels)))
        E = float(10.0 ** rng.uniform(0.0, 3.0))
        nu = float(rng.uniform(0.2, 0.45))
        amp = float(rng.uniform(0.5, 2.0))
        th = float(rng.uniform(0.0, 2.0 * math.pi))
        tx, ty = amp * math.cos(th), amp * math.sin(th)
        if q == 1:
            p = Problem(L=L, patches=[(0, 0)], E=E, nu=nu, bc=[(CLAMP, 0, 0, 0)],
                        traction=[(0, TOP, tx, ty)])
        elif q == 2:
            p = Problem(L=L, patches=[(0, 0), (1, 0)], E=E, nu=nu,
                        bc=[(CLAMP, 0, 0, 0), (0, 0, 0, 0)],
                        traction=[(0, TOP, tx, ty), (1, TOP, tx, ty)])
        else:
            p = Problem(L=L, patches=[(0, 0), (1, 0), (0, 1)], E=E, nu=nu,
                        bc=[(0, 0, CLAMP, 0), (0, 0, CLAMP, 0), (0, 0, 0, 0)],
                        traction=[(1, TOP, tx, ty), (2, TOP, tx, ty)])
        out.append(p)
    return out


# ----------------------------------------------------------------------------
# Random tensor-train data for kernel parity tests
# ----------------------------------------------------------------------------

def random_tt(seed: int, modes: Sequence[int], ranks: Sequence[int], scale: float = 1.0) -> List[np.ndarray]:
    """Random MPS cores of shape (r_{k-1}, n_k, r_k); ranks has len(modes)+1
    entries with ranks[0] = ranks[-1] = 1.  Entries are N(0, 1) * scale /
    sqrt(r_{k-1} n_k) so that the represented tensor stays O(1)."""
    assert len(ranks) == len(modes) + 1
    rng = np.random.default_rng(seed)
    cores = []
    for k, n in enumerate(modes):
        r0, r1 = ranks[k], ranks[k + 1]
        cores.append(rng.standard_normal((r0, n, r1)) * (scale / math.sqrt(r0 * n)))
    return cores


def random_mpo(seed: int, rows: Sequence[int], cols: Sequence[int], ranks: Sequence[int]) -> List[np.ndarray]:
    """Random MPO cores of shape (R_{k-1}, n_k, m_k, R_k)."""
    assert len(ranks) == len(rows) + 1 and len(rows) == len(cols)
    rng = np.random.default_rng(seed)
    cores = []
    for k in range(len(rows)):
        r0, r1 = ranks[k], ranks[k + 1]
        cores.append(rng.standard_normal((r0, rows[k], cols[k], r1)) / math.sqrt(r0 * cols[k]))
    return cores


def qtt_modes(prob: Problem) -> List[int]:
    """Mode sizes of the QTT layout: L position cores of mode 4, then a patch
    core of mode q (omitted when q = 1), then a component core of mode 2."""
    modes = [4] * prob.L
    if prob.q > 1:
        modes.append(prob.q)
    modes.append(2)
    return modes
