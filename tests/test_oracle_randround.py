"""Pins of the O-4 randomized residual rounding: the counter-based generator
against SplitMix64's published outputs and the normal law, exactness when the
sketch reaches the ranks of f - K u, the orthogonal-projection identity, and
left-orthonormal cores."""
import os

import numpy as np
import pytest
from scipy import stats

import workloads as W
from oracle import assembly, randround, tt

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_mix64_matches_published_splitmix64():
    want = [int(ln, 16) for ln in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if not ln.startswith("#")]
    gamma = 0x9E3779B97F4A7C15
    states = [(k * gamma) & ((1 << 64) - 1) for k in range(len(want))]
    assert [randround.mix64(s) for s in states] == want
    vec = randround.mix64(np.array(states, dtype=np.uint64))
    assert [int(v) for v in vec] == want


def test_gaussian_draws_follow_the_normal_law():
    g = randround.gaussian(12345, 200_000)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.02
    assert stats.kstest(g, "norm").pvalue > 1e-3
    # different keys give different streams, the same key the same one
    assert not np.allclose(g[:100], randround.gaussian(12346, 100))
    np.testing.assert_array_equal(g[:100], randround.gaussian(12345, 100))


def _problem(L=4):
    prob = W.plate_traction_smooth(L)
    K, f = assembly.assemble(prob)
    u = W.random_tt(23, W.qtt_modes(prob), [1] + [5] * (len(W.qtt_modes(prob)) - 1) + [1])
    y = tt.full(f) - tt.full_matrix(K) @ tt.full(u)
    return K, f, u, y


def test_full_sketch_rank_reproduces_the_residual():
    K, f, u, y = _problem()
    r, nr = randround.round_residual(K, u, f, ell=4096, seed=1)
    np.testing.assert_allclose(tt.full(r), y, rtol=0, atol=1e-12 * np.linalg.norm(y))
    assert nr == pytest.approx(np.linalg.norm(y), rel=1e-12)


@pytest.mark.parametrize("ell", [3, 10, 30])
def test_projection_identity_and_orthonormal_cores(ell):
    K, f, u, y = _problem()
    r, nr = randround.round_residual(K, u, f, ell=ell, seed=2)
    yr = tt.full(r)
    assert nr == pytest.approx(np.linalg.norm(yr), rel=1e-12)
    err2 = np.linalg.norm(y - yr) ** 2
    assert abs(err2 + nr ** 2 - np.linalg.norm(y) ** 2) <= 1e-10 * np.linalg.norm(y) ** 2
    for c in r[:-1]:
        m = c.reshape(-1, c.shape[2], order="F")
        np.testing.assert_allclose(m.T @ m, np.eye(m.shape[1]), atol=1e-12)
    assert max(tt.ranks(r)) <= ell


def test_error_shrinks_with_sketch_rank():
    K, f, u, y = _problem()
    errs = [np.linalg.norm(y - tt.full(randround.round_residual(K, u, f, ell=e, seed=3)[0])) for e in (2, 8, 32)]
    assert errs[0] > errs[1] > errs[2]
