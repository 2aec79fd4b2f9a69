"""Pins of the oracle's learned-guess pieces (features, samples, network,
gradient, AdamW) against closed forms, the exact inversion of Section 2.3,
central differences and library routines (torch autograd and torch.optim)."""
import math

import numpy as np
import pytest

import oracle as O

GAM = 13.0 / 9.0
FLAT = np.diag([-1.0, 1.0, 1.0, 1.0])
LOG_CLAMP = math.log(1e-30)


def _grid(n1=32, n2=32):
    return O.Grid(O.default_params(n1=n1, n2=n2, gam=GAM))


def _rand_theta(rng, scale=0.3):
    return (rng.standard_normal(O.MLP_NPARAM) * scale).astype(np.float32)


def _rand_norm(rng):
    return np.concatenate([rng.uniform(-1, 1, 5), rng.uniform(0.5, 2.0, 5), [0.3], [1.7]]).astype(np.float32)


# ------------------------------------------------------------------ rounding

def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.standard_normal(2000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 2000),
        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 1e-40, -3e-39, 3.0e38, 0.0],
                 dtype=np.float32),
    ]).astype(np.float32)
    # exact ties: lower 16 bits = 0x8000
    ties = (rng.integers(0, 2 ** 31, 200, dtype=np.int64) & ~0xFFFF | 0x8000).astype(np.uint32).view(np.float32)
    ties = ties[np.isfinite(ties)]
    x = np.concatenate([x, ties])
    ours = O.bf16_round(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))


# ------------------------------------------------------------------ features

def test_features_flat_rest_unmagnetised_closed_form():
    g = O.geom_from(FLAT)
    rho, u = 0.37, 0.05
    U = O.prim_to_U(np.array([rho, u, 0, 0, 0, 0, 0, 0.0]), g, GAM)
    f, rc = O.mlp_features(U, g)
    assert rc == 0
    # at rest: D = rho, tau = u, no momentum, no field
    assert f[0] == pytest.approx(math.log(u / rho), abs=1e-13)
    assert f[1] == LOG_CLAMP and f[2] == LOG_CLAMP and f[3] == LOG_CLAMP
    assert f[4] == pytest.approx(math.log(rho), abs=1e-15)


def test_features_flat_moving_unmagnetised_closed_form():
    g = O.geom_from(FLAT)
    rho, u, ux = 0.2, 0.7, 3.0
    U = O.prim_to_U(np.array([rho, u, ux, 0, 0, 0, 0, 0.0]), g, GAM)
    f, _ = O.mlp_features(U, g)
    lor = math.sqrt(1 + ux * ux)
    W = lor * lor * (rho + GAM * u)
    D = lor * rho
    v2 = 1 - 1 / lor ** 2
    p = (GAM - 1) * u
    # energy -n.Q = W - p; momentum squared W^2 v^2 (Section 2.3 with B = 0)
    assert f[0] == pytest.approx(math.log((W - p - D) / D), abs=1e-13)
    assert f[1] == pytest.approx(math.log(W * W * v2 / D ** 2), abs=1e-13)
    assert f[4] == pytest.approx(math.log(D), abs=1e-14)


def test_features_flat_rest_magnetised_closed_form():
    g = O.geom_from(FLAT)
    rho, u, B = 0.5, 0.1, np.array([0.3, -0.4, 1.2])
    U = O.prim_to_U(np.array([rho, u, 0, 0, 0, *B]), g, GAM)
    f, _ = O.mlp_features(U, g)
    B2 = float(B @ B)
    # static field: energy u + rho + B^2/2, Bf = B, Q_i = 0
    assert f[0] == pytest.approx(math.log((u + 0.5 * B2) / rho), abs=1e-13)
    assert f[2] == pytest.approx(math.log(B2 / rho), abs=1e-13)
    assert f[3] == LOG_CLAMP


def test_features_homogeneity_at_kerr_points():
    G = _grid()
    rng = np.random.default_rng(3)
    for i, j in [(0, 5), (3, 16), (20, 1), (31, 31)]:
        g = G.geom_at(G.x1in + (i + 0.5) * G.dx[0], G.x2in + (j + 0.5) * G.dx[1])
        q = np.array([0.3, 0.2, *rng.uniform(-0.5, 0.5, 3), *rng.uniform(-0.5, 0.5, 3)])
        U = O.prim_to_U(q, g, GAM)
        f, _ = O.mlp_features(U, g)
        lam = 7.3
        Us = U * lam
        Us[5:8] = U[5:8] * math.sqrt(lam)
        fs, _ = O.mlp_features(Us, g)
        assert np.allclose(fs[:4], f[:4], rtol=0, atol=1e-12)
        assert fs[4] == pytest.approx(f[4] + math.log(lam), abs=1e-13)


def test_features_reject_nonpositive_density():
    g = O.geom_from(FLAT)
    U = O.prim_to_U(np.array([0.3, 0.1, 0, 0, 0, 0, 0, 0.0]), g, GAM)
    U[0] = -1.0
    f, rc = O.mlp_features(U, g)
    assert rc == -1 and np.all(f == 0)


# ------------------------------------------------------------------ samples

def test_samples_follow_the_stated_distribution():
    G = _grid(24, 40)
    seed, n = 7, 400
    P, loc, U, feat, lab = G.mlp_samples(seed, 0, n)
    for a in range(n):
        xi = [O.uniform(seed, 16 * a + k) for k in range(10)]
        i1, j1 = min(int(xi[0] * 24), 23), min(int(xi[1] * 40), 39)
        assert loc[a] == i1 * 40 + j1
        assert P[0, a] == pytest.approx(1e-6 ** (1 - xi[2]), rel=1e-13)
        assert P[1, a] / P[0, a] == pytest.approx(1e-4 * 1e5 ** xi[3], rel=1e-13)
        g = G.geom_at(G.x1in + (i1 + 0.5) * G.dx[0], G.x2in + (j1 + 0.5) * G.dx[1])
        s, _ = O.state_of(P[:, a], g)
        # b^2 carries the cancellation of (B^2 + (B.u)^2)/(u^t)^2 at Gamma up to 50
        assert s["gamma"] == pytest.approx(50.0 ** xi[4], rel=1e-12)
        assert s["bsq"] / P[0, a] == pytest.approx(1e-3 * 1e5 ** xi[5], rel=1e-10)
    assert P[0].min() >= 1e-6 and P[0].max() <= 1.0
    # deterministic in the seed, different across seeds
    P2 = G.mlp_samples(seed, 10, 5)[0]
    assert np.array_equal(P2, P[:, 10:15])
    assert not np.allclose(G.mlp_samples(seed + 1, 0, 5)[0], P[:, :5])


def test_sample_labels_match_the_exact_inversion():
    G = _grid()
    n = 3000
    P, loc, U, feat, lab = G.mlp_samples(11, 0, n)
    # start Newton far away: a static guess of the right density scale
    guess = np.zeros_like(P)
    guess[0] = 1.0
    guess[1] = 1.0
    Pr, flags, it = G.con2prim(U, loc, guess, methods=15)
    ok = (flags & O.C2P_FAIL) == 0
    assert ok.mean() > 0.95
    for a in np.nonzero(ok)[0][:800]:
        i1, j1 = divmod(int(loc[a]), G.p.n2)
        g = G.geom_at(G.x1in + (i1 + 0.5) * G.dx[0], G.x2in + (j1 + 0.5) * G.dx[1])
        s, _ = O.state_of(Pr[:, a], g)
        W = s["gamma"] ** 2 * (Pr[0, a] + GAM * Pr[1, a])
        D = g.alpha * U[0, a] / g.gdet
        assert math.log(W / D) == pytest.approx(lab[a], abs=1e-8)
        f, _ = O.mlp_features(U[:, a], g)
        assert np.array_equal(f, feat[:, a])


def test_learned_start_reaches_the_same_root():
    G = _grid()
    n = 500
    P, loc, U, feat, lab = G.mlp_samples(5, 0, n)
    D = np.zeros(n)
    for a in range(n):
        i1, j1 = divmod(int(loc[a]), G.p.n2)
        g = G.geom_at(G.x1in + (i1 + 0.5) * G.dx[0], G.x2in + (j1 + 0.5) * G.dx[1])
        D[a] = g.alpha * U[0, a] / g.gdet
    guess = P * (1 + 0.3 * np.sin(np.arange(n)))[None, :]
    Pa, fa, ia = G.con2prim(U, loc, guess)
    # a starting W within 1e-3 of the root: same root, fewer Newton steps
    Wg = D * np.exp(lab) * (1 + 1e-3)
    Pb, fb, ib = G.con2prim_w(U, loc, guess, Wg)
    # the method choice (Newton, or the beta < 1e-2 entropy switch of the
    # guess primitives) does not depend on the starting W
    assert np.array_equal(fa, fb)
    both = fa == O.C2P_NR
    assert both.mean() > 0.5
    assert np.allclose(Pb[:, both], Pa[:, both], rtol=1e-9, atol=1e-14)
    assert ib[both].mean() < ia[both].mean()
    # wguess <= 0 is the plain start
    Pc, fc, ic = G.con2prim_w(U, loc, guess, np.zeros(n))
    assert np.array_equal(Pc, Pa) and np.array_equal(ic, ia)


# ------------------------------------------------------------------ network

def test_forward_of_hand_built_network():
    th = np.zeros(O.MLP_NPARAM, dtype=np.float32)
    W1 = th[0:320].reshape(64, 5)
    W1[0, 0], W1[1, 0] = 1.0, -1.0
    W2 = th[384:4480].reshape(64, 64)
    W2[0, 0] = 1.0 + 2.0 ** -10          # rounds to 1 in BF16
    W2[1, 1] = 1.0
    W3 = th[4544:4608]
    W3[0], W3[1] = 1.0, -1.0
    norm = np.array([0.5, 0, 0, 0, 0, 2.0, 1, 1, 1, 1, 0.25, 3.0], dtype=np.float32)
    f = np.random.default_rng(1).uniform(-5, 5, (5, 50)).astype(np.float32)
    y = O.mlp_forward(th, norm, f)
    # relu(x) - relu(-x) = x: the network returns its standardised first input
    x0 = (f[0].astype(np.float64) - 0.5) / 2.0
    assert np.allclose(y, x0 * 3.0 + 0.25, rtol=0, atol=1e-14)
    # a bias is not rounded
    th2 = th.copy()
    th2[4608] = 1.0 + 2.0 ** -12
    y2 = O.mlp_forward(th2, norm, f)
    assert np.allclose(y2 - y, 3.0 * 2.0 ** -12 + 3.0, rtol=0, atol=1e-12)


def _feat_batch(rng, n):
    f = rng.standard_normal((5, n)).astype(np.float32)
    lab = rng.uniform(0, 4, n).astype(np.float32)
    return f, lab


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    w = rng.standard_normal(O.MLP_NPARAM) * 0.3
    norm = _rand_norm(rng)
    f, lab = _feat_batch(rng, 24)
    L0, g = O.mlp_loss_grad_exact(w, norm, f, lab)
    idx = np.concatenate([rng.choice(np.arange(a, b), min(12, b - a), replace=False)
                          for a, b in O.MLP_SLICES.values()])
    h = 1e-6
    for k in idx:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (O.mlp_loss_grad_exact(wp, norm, f, lab)[0] - O.mlp_loss_grad_exact(wm, norm, f, lab)[0]) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-6, abs=1e-9)


def _torch_net(torch, w, norm, f, lab, bf16_forward):
    """The same network written with torch tensors (float64)."""
    tw = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    if bf16_forward:
        eff = tw.to(torch.float32).to(torch.bfloat16).to(torch.float64)
        mask = torch.ones(O.MLP_NPARAM, dtype=torch.bool)
        for name in ("b1", "b2", "b3"):
            a, b = O.MLP_SLICES[name]
            mask[a:b] = False
        # w holds FP32 values already; biases enter unrounded
        weff = torch.where(mask, tw + (eff - tw).detach(), tw)
    else:
        weff = tw
    sl = {k: weff[a:b] for k, (a, b) in O.MLP_SLICES.items()}
    nm = torch.tensor(norm, dtype=torch.float64)
    x = (torch.tensor(f, dtype=torch.float64).T - nm[:5]) / nm[5:10]
    h1 = torch.relu(x @ sl["W1"].reshape(64, 5).T + sl["b1"])
    h2 = torch.relu(h1 @ sl["W2"].reshape(64, 64).T + sl["b2"])
    s = h2 @ sl["W3"] + sl["b3"]
    t = (torch.tensor(lab, dtype=torch.float64) - nm[10]) / nm[11]
    loss = ((s - t) ** 2).mean()
    return tw, loss


def test_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    th = _rand_theta(rng)
    norm = _rand_norm(rng)
    f, lab = _feat_batch(rng, 64)
    L, g = O.mlp_loss_grad(th, norm, f, lab)
    tw, loss = _torch_net(torch, th.astype(np.float64), norm, f, lab, bf16_forward=True)
    loss.backward()
    assert L == pytest.approx(loss.item(), rel=1e-13)
    assert np.allclose(g, tw.grad.numpy(), rtol=1e-11, atol=1e-14)


def test_adamw_first_step_closed_form():
    rng = np.random.default_rng(5)
    th0 = rng.standard_normal(O.MLP_NPARAM)
    g = rng.standard_normal(O.MLP_NPARAM) * 1e-3
    th, m, v = th0.copy(), np.zeros_like(th0), np.zeros_like(th0)
    lr, wd, eps = 1e-2, 0.1, 1e-8
    O.mlp_adamw(th, m, v, g, 1, lr, 0.9, 0.999, eps, wd)
    decay = np.zeros(O.MLP_NPARAM, dtype=bool)
    for name in ("W1", "W2", "W3"):
        a, b = O.MLP_SLICES[name]
        decay[a:b] = True
    # bias-corrected moments equal g and g^2 after one step
    expect = np.where(decay, th0 * (1 - lr * wd), th0) - lr * g / (np.abs(g) + eps)
    assert np.allclose(th, expect, rtol=1e-14, atol=1e-16)


def test_adamw_matches_torch_optim():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    th0 = rng.standard_normal(O.MLP_NPARAM)
    th, m, v = th0.copy(), np.zeros_like(th0), np.zeros_like(th0)
    decay = np.zeros(O.MLP_NPARAM, dtype=bool)
    for name in ("W1", "W2", "W3"):
        a, b = O.MLP_SLICES[name]
        decay[a:b] = True
    pd = torch.tensor(th0[decay], dtype=torch.float64, requires_grad=True)
    pn = torch.tensor(th0[~decay], dtype=torch.float64, requires_grad=True)
    opt = torch.optim.AdamW([{"params": [pd], "weight_decay": 0.05}, {"params": [pn], "weight_decay": 0.0}],
                            lr=3e-3, betas=(0.8, 0.99), eps=1e-7)
    for step in range(1, 6):
        g = rng.standard_normal(O.MLP_NPARAM)
        O.mlp_adamw(th, m, v, g, step, 3e-3, 0.8, 0.99, 1e-7, 0.05)
        pd.grad = torch.tensor(g[decay])
        pn.grad = torch.tensor(g[~decay])
        opt.step()
    ref = np.zeros(O.MLP_NPARAM)
    ref[decay] = pd.detach().numpy()
    ref[~decay] = pn.detach().numpy()
    assert np.allclose(th, ref, rtol=1e-13, atol=1e-15)


def test_train_steps_match_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    th0 = _rand_theta(rng, 0.2)
    norm = _rand_norm(rng)
    f, lab = _feat_batch(rng, 40)
    batch, nsteps, lr, wd = 16, 4, 1e-3, 0.01
    th, loss = O.mlp_train_steps(th0, norm, f, lab, batch, nsteps, lr, wd=wd)
    # torch: the same batches, the same straight-through BF16 forward, AdamW
    w = th0.astype(np.float64)
    decay = np.zeros(O.MLP_NPARAM, dtype=bool)
    for name in ("W1", "W2", "W3"):
        a, b = O.MLP_SLICES[name]
        decay[a:b] = True
    mom = np.zeros(O.MLP_NPARAM)
    vel = np.zeros(O.MLP_NPARAM)
    for s in range(nsteps):
        idx = (s * batch + np.arange(batch)) % f.shape[1]
        tw, ls = _torch_net(torch, w.astype(np.float32).astype(np.float64), norm, f[:, idx], lab[idx], True)
        ls.backward()
        g = tw.grad.numpy()
        w = w.copy()
        O.mlp_adamw(w, mom, vel, g, s + 1, lr, 0.9, 0.999, 1e-8, wd)
        last = ls.item()
    assert loss == pytest.approx(last, rel=1e-12)
    assert np.allclose(th, w.astype(np.float32), rtol=2e-7, atol=1e-9)
