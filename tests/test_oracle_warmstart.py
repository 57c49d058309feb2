"""Pins of the warm-start oracle: the analytic MLP backward and the TT-loss
gradient against central finite differences, and the gauge invariance of the
loss (multiplying one core by G and the next by G^-1 leaves it unchanged)."""
import numpy as np

import workloads as W
from oracle import tt, warmstart as ws


def test_tt_loss_value_and_gauge_invariance():
    modes = [4, 4, 4, 2]
    X = W.random_tt(1, modes, [1, 3, 5, 2, 1])
    Xh = W.random_tt(2, modes, [1, 4, 4, 2, 1])
    loss, _ = ws.tt_loss_and_grad(Xh, X)
    ref = np.linalg.norm(tt.full(Xh) - tt.full(X)) ** 2 / np.linalg.norm(tt.full(X)) ** 2
    assert abs(loss - ref) <= 1e-12 * max(1.0, ref)
    G = np.random.default_rng(0).standard_normal((4, 4)) + 3 * np.eye(4)
    Xg = [c.copy() for c in Xh]
    Xg[1] = np.einsum("aib,bc->aic", Xg[1], G)
    Xg[2] = np.einsum("ab,bic->aic", np.linalg.inv(G), Xg[2])
    lg, _ = ws.tt_loss_and_grad(Xg, X)
    assert abs(lg - loss) <= 1e-10 * max(1.0, loss)


def test_tt_loss_gradient_finite_difference():
    modes = [4, 4, 2]
    X = W.random_tt(3, modes, [1, 3, 2, 1])
    Xh = W.random_tt(4, modes, [1, 2, 2, 1])
    _, g = ws.tt_loss_and_grad(Xh, X)
    rng = np.random.default_rng(5)
    for k in range(3):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in Xh[k].shape)
            h = 1e-6
            Xp = [c.copy() for c in Xh]; Xp[k][idx] += h
            Xm = [c.copy() for c in Xh]; Xm[k][idx] -= h
            fd = (ws.tt_loss_and_grad(Xp, X)[0] - ws.tt_loss_and_grad(Xm, X)[0]) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(1.0, abs(fd))


def test_mlp_backward_finite_difference():
    modes = [4, 4, 2]
    r = 2
    P = ws.n_outputs(modes, r)
    p = ws.init_params(0, 4, 8, P, out_scale=0.5)
    params = W.plate_params(7, 3)
    phi = ws.features(params)
    targets = [W.random_tt(10 + b, modes, [1, 3, 2, 1]) for b in range(3)]

    def L(pp):
        o, _ = ws.forward(pp, phi)
        return ws.batch_loss_and_grad(o, targets, modes, r)[0]

    o, cache = ws.forward(p, phi)
    _, go = ws.batch_loss_and_grad(o, targets, modes, r)
    g = ws.backward(p, cache, go)
    rng = np.random.default_rng(1)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in p[name].shape)
            h = 1e-6
            pp = {k: v.copy() for k, v in p.items()}; pp[name][idx] += h
            pm = {k: v.copy() for k, v in p.items()}; pm[name][idx] -= h
            fd = (L(pp) - L(pm)) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-5 * max(1e-3, abs(fd)), (name, fd, g[name][idx])


def test_output_count_matches_plate_layout():
    """Rank-16 cores for the L = 12 plate: 4 x 16 + 11 x 16 x 4 x 16 + 16 x 2."""
    assert ws.n_outputs([4] * 12 + [2], 16) == 64 + 11 * 1024 + 32 == 11360


def _adam_run(grads, lr=0.01, p0=0.0):
    p = {"w": np.array([p0])}
    state = {}
    out = []
    for t, g in enumerate(grads, start=1):
        ws.adam_step(p, {"w": np.array([g])}, state, lr=lr, t=t)
        out.append(float(p["w"][0]))
    return out


def test_adam_first_step_and_constant_gradient_move_by_lr():
    """Kingma & Ba (2015), Sec. 2.1 and Alg. 1: with bias correction the first
    update is lr * g / (|g| + eps), whatever |g|; under a constant gradient
    m_hat = g and v_hat = g^2 at every step, so every step moves by the same
    amount.  A wrong bias-correction power or swapped beta1/beta2 breaks
    both."""
    eps = 1e-8
    for g in (3.7, -0.02, 250.0):
        traj = _adam_run([g] * 5, lr=0.01)
        step = 0.01 * abs(g) / (abs(g) + eps)
        moves = np.diff([0.0] + traj)
        np.testing.assert_allclose(moves, -np.sign(g) * step, rtol=1e-12)


def test_adam_two_steps_by_hand():
    """Gradients +1 then -1 with beta1 = 0.9, beta2 = 0.999 (Alg. 1 defaults),
    worked by hand: m_1 = 0.1, v_1 = 0.001, m_hat_1 = 1, v_hat_1 = 1;
    m_2 = 0.09 - 0.1 = -0.01, m_hat_2 = -0.01 / 0.19 = -1/19;
    v_2 = 0.000999 + 0.001 = 0.001999, v_hat_2 = 0.001999 / (1 - 0.998001) = 1.
    So p_1 = -lr / (1 + eps) and p_2 = p_1 + lr / (19 (1 + eps))."""
    lr, eps = 0.01, 1e-8
    p1, p2 = _adam_run([1.0, -1.0], lr=lr)
    assert abs(p1 - (-lr / (1 + eps))) <= 1e-15
    assert abs(p2 - (p1 + lr / (19.0 * (1 + eps)))) <= 1e-15


def test_adam_invariant_to_gradient_scale():
    """The update is invariant to a positive rescaling of the gradients
    (Kingma & Ba, Sec. 2.1), up to the eps term."""
    rng = np.random.default_rng(3)
    gs = rng.standard_normal(6)
    a = _adam_run(list(gs), lr=0.05)
    b = _adam_run(list(1e3 * gs), lr=0.05)
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-9)
