"""Learned warm start on the GPU: the project's forward, loss and backward
kernels against the NumPy oracle (FP32 tolerance), and what the trained
network gains over a cold start on a small plate level."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import tt, warmstart as ows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2501_07778_gb300 as q  # noqa: E402
from paper_2501_07778_gb300 import warmstart as ws  # noqa: E402


def _to_gpu(p):
    # oracle matrices act as W @ x; column-major (rows x cols) = torch (cols, rows)
    return {"W1": torch.tensor(p["W1"].T, dtype=torch.float32).contiguous().cuda(),
            "b1": torch.tensor(p["b1"], dtype=torch.float32).cuda(),
            "W2": torch.tensor(p["W2"].T, dtype=torch.float32).contiguous().cuda(),
            "b2": torch.tensor(p["b2"], dtype=torch.float32).cuda(),
            "W3": torch.tensor(p["W3"].T, dtype=torch.float32).contiguous().cuda(),
            "b3": torch.tensor(p["b3"], dtype=torch.float32).cuda()}


def test_forward_loss_backward_match_oracle():
    modes, r, H = [4, 4, 4, 2], 3, 16
    P = ows.n_outputs(modes, r)
    op = ows.init_params(3, 4, H, P, out_scale=0.5)
    op["b1"] = np.random.default_rng(1).standard_normal(H) * 0.1
    op["b3"] = np.random.default_rng(2).standard_normal(P) * 0.05
    net = ws.WarmStartMLP(modes, r=r, H=H)
    net.params = _to_gpu(op)
    params = W.plate_params(4, 5)
    basis_np = [W.random_tt(20 + t, modes, [1, 3, 4, 2, 1]) for t in range(4)]
    basis = [q.QTT.from_cores(b, prec=q.QTT_F32) for b in basis_np]
    coef = np.random.default_rng(7).standard_normal((5, 4))
    coef[:, 2:] = 0.0                       # sparse combinations, as in training
    phi_np = ows.features(params)
    phi = torch.tensor(phi_np, dtype=torch.float32).cuda()
    out, h1, h2 = net.forward(phi)
    o_ref, cache = ows.forward(op, phi_np)
    np.testing.assert_allclose(out.cpu().numpy(), o_ref, rtol=2e-4, atol=2e-5)
    targets = []
    for b in range(5):
        acc = None
        for t in range(4):
            if coef[b, t] != 0.0:
                term = tt.scale(basis_np[t], coef[b, t])
                acc = term if acc is None else tt.add(acc, term)
        targets.append(acc)
    loss, gout = net.loss_and_grad(out, basis, coef)
    l_ref, go_ref = ows.batch_loss_and_grad(out.double().cpu().numpy(), targets, modes, r)
    assert float(loss.mean()) == pytest.approx(l_ref, rel=1e-4)
    np.testing.assert_allclose(gout.cpu().numpy(), go_ref, rtol=2e-3, atol=1e-5 * np.abs(go_ref).max())
    g = net.backward(phi, h1, h2, gout)
    g_ref = ows.backward(op, cache, go_ref)
    for k in ("W1", "W2", "W3"):
        np.testing.assert_allclose(g[k].cpu().numpy(), g_ref[k].T, rtol=3e-3, atol=1e-5 * np.abs(g_ref[k]).max())
    for k in ("b1", "b2", "b3"):
        np.testing.assert_allclose(g[k].cpu().numpy(), g_ref[k], rtol=3e-3, atol=1e-5 * np.abs(g_ref[k]).max())


def test_adam_matches_oracle():
    n = 1000
    w = torch.randn(n, device="cuda")
    gg = torch.randn(n, device="cuda")
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    ref = {"w": w.double().cpu().numpy().copy()}
    st = {}
    for t in (1, 2):
        q.lib().qtt_ws_adam(n, ws._p(w), ws._p(gg), ws._p(m), ws._p(v), 1e-2, 0.9, 0.999, 1e-8, t, None)
        ows.adam_step(ref, {"w": gg.double().cpu().numpy()}, st, 1e-2, t)
    torch.cuda.synchronize()
    np.testing.assert_allclose(w.cpu().numpy(), ref["w"], rtol=1e-5, atol=1e-6)


def test_trained_warm_start_beats_cold_start():
    """Train on superpositions of method solves at L = 5 and compare the
    sweeps a held-out solve needs from the predicted start and from a cold
    (rank-1) start."""
    L = 5
    nus = [0.2, 0.3, 0.4, 0.45]
    basis64 = ws.basis_solutions(L, nus, tol=1e-9)
    basis = [b.copy(prec=q.QTT_F32) for b in basis64]
    modes = W.qtt_modes(W.plate_top_traction(L, 1.0, 0.3, 1.0, 0.0))
    net = ws.WarmStartMLP(modes, r=8, H=64, seed=0)
    P, coef = ws.dataset(1, 256, nus)
    losses = []
    for step in range(300):
        idx = np.random.default_rng(step).integers(0, len(P), 32)
        losses.append(net.train_step(P[idx], basis, coef[idx], lr=2e-3))
    assert np.mean(losses[-20:]) < 0.2 * np.mean(losses[:5])
    held = W.plate_params(2, 3)
    held[:, 1] = np.clip(held[:, 1], 0.2, 0.45)
    x0s = net.predict(held)
    warm, cold = 0, 0
    for b in range(3):
        E, nu, amp, th = held[b]
        K, f = q.qtt_assemble_stiffness(W.plate_top_traction(L, E, nu, amp, th))
        _, iw = q.qtt_solve(K, f, x0s[b], tol=1e-9, kick_rank=4)
        _, ic = q.qtt_solve(K, f, tol=1e-9, kick_rank=4)
        assert iw["rel_residual"] <= 1e-8 and ic["rel_residual"] <= 1e-8
        warm += iw["sweeps"]
        cold += ic["sweeps"]
    assert warm < cold, (warm, cold)


def test_superposition_start_is_accurate_in_the_residual():
    """The non-learned start (stored unit-traction solutions interpolated in
    nu, scaled by amp / E) has a small relative residual, the solve from it
    reaches the sparse direct solution, and it needs fewer sweeps than a
    cold start."""
    import workloads as W
    from oracle import fem
    from paper_2501_07778_gb300 import warmstart as ws
    L = 7
    ss = ws.SuperpositionStart(L, (0.2, 0.3, 0.4, 0.45), order=3, tol=1e-10, precision=q.QTT_MIXED, kick_rank=8)
    P = W.plate_params(2, 3)
    x0s = ss.predict(P)
    for (E, nu, amp, th), x0 in zip(P, x0s):
        prob = W.plate_top_traction(L, float(E), float(nu), float(amp), float(th))
        K, f = q.qtt_assemble_stiffness(prob)
        r0 = q.qtt_residual_fe(K, x0, f)
        assert r0 <= 0.05, r0
        u, info = q.qtt_solve(K, f, x0=x0, tol=1e-9, precision=q.QTT_MIXED, kick_rank=8, max_sweeps=30)
        uc, ic = q.qtt_solve(K, f, tol=1e-9, precision=q.QTT_MIXED, kick_rank=8, max_sweeps=30)
        assert info["rc"] == 0 and ic["rc"] == 0
        assert info["sweeps"] <= ic["sweeps"], (info["sweeps"], ic["sweeps"])
        um, nm = fem.solve_merged(prob)
        ref = fem.merged_to_qtt(prob, um, nm)
        ug = q.qtt_to_full(u).cpu().numpy()
        assert np.linalg.norm(ug - ref) / np.linalg.norm(ref) <= 1e-7
