"""GPU parity of the core TT operations (through the C ABI) against the
oracle: full expansion in both orderings (bit-exact permutation), the MPO x
MPS product, sums, norms, rounding and the FP64 residual.  Shapes span
several GEMM tiles with ragged tails (ranks not multiples of 64)."""
import numpy as np
import pytest

import workloads as W
from oracle import indexing, tt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2501_07778_gb300 as q  # noqa: E402


def _full(x, ordering=q.QTT_ORDER_Z_BLOCK):
    return q.qtt_to_full(x, ordering).cpu().numpy()


@pytest.mark.parametrize("modes,ranks", [([4, 4, 4, 2], [1, 3, 7, 2, 1]),
                                         ([4, 4, 4, 4, 4, 3, 2], [1, 4, 16, 37, 70, 6, 2, 1]),
                                         ([5], [1, 1])])
def test_to_full_matches_oracle(modes, ranks):
    cores = W.random_tt(1, modes, ranks)
    x = q.QTT.from_cores(cores)
    assert x.ranks == ranks
    np.testing.assert_allclose(_full(x), tt.full(cores), rtol=1e-13, atol=1e-14)
    back = x.cores()
    for a, b in zip(back, cores):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("L,qq", [(3, 1), (4, 3), (2, 2)])
def test_to_full_canonical_is_exact_permutation(L, qq):
    modes = [4] * L + ([qq] if qq > 1 else []) + [2]
    cores = W.random_tt(2, modes, [1] + [3] * (len(modes) - 1) + [1])
    x = q.QTT.from_cores(cores)
    z = _full(x, q.QTT_ORDER_Z_BLOCK)
    c = _full(x, q.QTT_ORDER_CANONICAL)
    n = 1 << L
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for m in range(qq):
        for comp in range(2):
            src = indexing.qtt_dof(ii, jj, m, comp, L, qq)
            dst = indexing.canonical_dof(ii, jj, m, comp, L, qq)
            np.testing.assert_array_equal(c[dst.ravel()], z[src.ravel()])


def test_mpo_to_full_dense():
    A = W.random_mpo(3, [4, 4, 2], [4, 4, 2], [1, 5, 3, 1])
    x = q.QTT.from_cores(A)
    M = q.qtt_to_full(x).cpu().numpy().reshape(32, 32, order="F")
    np.testing.assert_allclose(M, tt.full_matrix(A), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("Rr", [((1, 5, 9, 4, 1), (1, 3, 11, 6, 1)), ((1, 16, 51, 43, 4, 1), (1, 4, 16, 30, 8, 1))])
def test_matvec_matches_oracle(Rr):
    R, r = Rr
    d = len(R) - 1
    modes = [4] * (d - 1) + [2]
    A = W.random_mpo(4, modes, modes, list(R))
    X = W.random_tt(5, modes, list(r))
    y = q.qtt_matvec(q.QTT.from_cores(A), q.QTT.from_cores(X))
    assert y.ranks == [a * b for a, b in zip(R, r)]
    ref = tt.full(tt.matvec(A, X))
    np.testing.assert_allclose(_full(y), ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_axpby_norm_residual():
    modes = [4, 4, 4, 2]
    X = W.random_tt(6, modes, [1, 4, 9, 2, 1])
    Y = W.random_tt(7, modes, [1, 3, 5, 2, 1])
    x, y = q.QTT.from_cores(X), q.QTT.from_cores(Y)
    z = q.qtt_axpby(2.0, x, -0.5, y)
    ref = 2.0 * tt.full(X) - 0.5 * tt.full(Y)
    np.testing.assert_allclose(_full(z), ref, rtol=1e-13, atol=1e-14)
    assert q.qtt_norm(z) == pytest.approx(np.linalg.norm(ref), rel=1e-12)
    A = W.random_mpo(8, modes, modes, [1, 3, 4, 2, 1])
    Ad = tt.full_matrix(A)
    res = q.qtt_residual(q.QTT.from_cores(A), x, y)
    ref_res = np.linalg.norm(tt.full(Y) - Ad @ tt.full(X)) / np.linalg.norm(tt.full(Y))
    assert res == pytest.approx(ref_res, rel=1e-10)


@pytest.mark.parametrize("eps", [1e-12, 1e-6, 1e-2])
def test_round_bound_and_ranks(eps):
    modes = [4, 4, 4, 4, 4, 2]
    X = W.random_tt(9, modes, [1, 4, 13, 30, 8, 2, 1])
    x = q.QTT.from_cores(X)
    xx = q.qtt_axpby(1.0, x, 1.0, x)
    q.qtt_round(xx, eps)
    ref = 2 * tt.full(X)
    err = np.linalg.norm(_full(xx) - ref)
    assert err <= max(eps, 1e-13) * np.linalg.norm(ref) * 1.001
    oracle = tt.round_tt(tt.add(X, X), eps)
    if eps <= 1e-6:
        assert xx.ranks == tt.ranks(oracle) == tt.ranks(X)
    else:
        # near the threshold the kept rank may differ by rounding of the tail
        assert all(abs(a - b) <= 2 for a, b in zip(xx.ranks, tt.ranks(oracle)))


def test_round_noisy_tensor_matches_oracle_ranks():
    rng = np.random.default_rng(3)
    v = rng.standard_normal(4 ** 5 * 2) * np.exp(-np.arange(4 ** 5 * 2) / 300.0)
    modes = [4] * 5 + [2]
    X = tt.tt_svd(v, modes, 1e-15)
    x = q.QTT.from_cores(X)
    for eps in (1e-1, 1e-3):
        y = x.copy()
        q.qtt_round(y, eps)
        o = tt.round_tt(X, eps)
        assert all(abs(a - b) <= 1 for a, b in zip(y.ranks, tt.ranks(o)))
        assert np.linalg.norm(_full(y) - v) <= eps * np.linalg.norm(v) * 1.001


def test_round_mpo_and_rank_cap():
    A = W.random_mpo(10, [4, 4, 2], [4, 4, 2], [1, 6, 3, 1])
    a = q.QTT.from_cores(A)
    aa = q.qtt_axpby(1.0, a, 1.0, a)
    q.qtt_round(aa, 1e-13)
    assert aa.ranks == [1, 6, 3, 1]
    M = q.qtt_to_full(aa).cpu().numpy().reshape(32, 32, order="F")
    np.testing.assert_allclose(M, 2 * tt.full_matrix(A), rtol=1e-12, atol=1e-13)
    b = q.qtt_axpby(1.0, a, 1.0, a)
    rc = q.qtt_round(b, 1e-13, max_rank=2)
    assert rc == -6 and max(b.ranks) == 2


def test_float32_path():
    modes = [4, 4, 4, 2]
    X = W.random_tt(11, modes, [1, 4, 9, 2, 1])
    x = q.QTT.from_cores(X, prec=q.QTT_F32)
    np.testing.assert_allclose(_full(x), tt.full(X), rtol=1e-5, atol=1e-6)
    xx = q.qtt_axpby(1.0, x, 1.0, x)
    q.qtt_round(xx, 1e-5)
    assert xx.ranks == [1, 4, 8, 2, 1]      # bond 2 is at most min(16, 8)
    np.testing.assert_allclose(_full(xx), 2 * tt.full(X), rtol=1e-4, atol=1e-5)
