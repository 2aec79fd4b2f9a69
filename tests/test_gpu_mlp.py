"""The learned Newton start on the GPU (C ABI) against the oracle:
- training samples;
- the BF16-weight forward pass;
- the FP32 gradient, held to 1e-5 relative of the FP64 backprop;
- short AdamW runs;
- a full training run whose guess leaves the inversion's root unchanged.

Sizes span several thread blocks plus a ragged tail.
"""
import numpy as np
import pytest

import oracle as O
from tests.gpu_common import gpu_mod, make_pair

pytestmark = pytest.mark.gpu
GAM = 13.0 / 9.0


def _pair(n1=24, n2=40):
    return make_pair(n1, n2, 1, gam=GAM)


def _rand_theta(rng, scale=0.3):
    return (rng.standard_normal(O.MLP_NPARAM) * scale).astype(np.float32)


def _norm_of(feat, lab):
    f = feat.astype(np.float64)
    return np.concatenate([f.mean(1), f.std(1) + 1e-3, [lab.mean()], [lab.std()]]).astype(np.float32)


@pytest.mark.parametrize("first,n", [(0, 20000), (123457, 777)])
def test_samples_match_oracle(first, n):
    G = gpu_mod()
    og, ctx = _pair()
    Pg, lg, Ug, fg, yg = G.mlp_samples(ctx, 7, first, n)
    Po, lo, Uo, fo, yo = og.mlp_samples(7, first, n)
    assert np.array_equal(lg, lo)
    # libm and CUDA's exp/log/sin/cos differ in the last bit: relative 1e-12;
    # the field is scaled by sqrt(sigma rho / b^2), and b^2 = (B^2 + (B.u)^2)/(u^t)^2
    # at Gamma up to 50 with the Kerr-Schild shift carries more of that rounding
    assert np.abs(Pg[:2] / Po[:2] - 1).max() < 1e-12
    for sl, tol in ((slice(2, 5), 1e-12), (slice(5, 8), 1e-11)):
        rel = np.linalg.norm(Pg[sl] - Po[sl], axis=0) / np.linalg.norm(Po[sl], axis=0)
        assert rel.max() < tol
    # T^t_nu cancels terms of size Gamma^2 (w + b^2): rounding times that
    # conditioning, as for the batched prim2cons
    xi = np.array([[O.uniform(7, 16 * (first + a) + k) for k in (4, 5)] for a in range(n)])
    cond = (50.0 ** xi[:, 0]) ** 2 * (1.0 + 1e-3 * 1e5 ** xi[:, 1])
    scaleU = np.abs(Uo[1:5]).max(0)
    assert np.abs(Ug[0] / Uo[0] - 1).max() < 1e-12
    assert (np.abs(Ug[1:5] - Uo[1:5]).max(0) / scaleU / (2.2e-16 * cond)).max() < 1e3
    assert (np.abs(Ug[8] / Uo[8] - 1) / (2.2e-16 * cond)).max() < 1e3
    # features and labels are the FP64 values rounded once to FP32; where the
    # argument cancels (tau = -n.Q - D at u/rho ~ 1e-4) the FP64 values carry
    # the cancellation, so allow a few FP32 ulps
    fo32 = fo.astype(np.float32)
    assert (np.abs(fg - fo32) <= 4e-7 * np.maximum(1.0, np.abs(fo32))).all()
    assert (np.abs(yg - yo.astype(np.float32)) <= 4e-7 * np.maximum(1.0, np.abs(yo))).all()


def test_load_get_and_forward_match_oracle():
    G = gpu_mod()
    og, ctx = _pair()
    rng = np.random.default_rng(0)
    _, _, _, f, y = G.mlp_samples(ctx, 3, 0, 5003)
    th = _rand_theta(rng)
    nm = _norm_of(f, y)
    G.mlp_load(ctx, th, nm)
    th2, nm2 = G.mlp_get(ctx)
    assert np.array_equal(th2, th) and np.array_equal(nm2, nm)
    yg = G.mlp_forward(ctx, f).astype(np.float64)
    yo = O.mlp_forward(th, nm, f)
    scale = np.abs(yo).max()
    # FP32 accumulation of 64-term dot products
    assert np.abs(yg - yo).max() <= 1e-5 * scale


def test_gradient_matches_oracle_backprop():
    G = gpu_mod()
    og, ctx = _pair()
    rng = np.random.default_rng(1)
    _, _, _, f, y = G.mlp_samples(ctx, 5, 0, 3000)   # 23 blocks of 128 and a tail of 56
    nm = _norm_of(f, y)
    for scale in (0.3, 0.1):
        th = _rand_theta(rng, scale)
        lg, gg = G.mlp_loss_grad(ctx, th, nm, f, y)
        lo, go = O.mlp_loss_grad(th, nm, f, y)
        assert lg == pytest.approx(lo, rel=1e-6)
        for name, (a, b) in O.MLP_SLICES.items():
            err = np.linalg.norm(gg[a:b] - go[a:b]) / np.linalg.norm(go[a:b])
            assert err < 1e-5, name


def test_gradient_of_single_sample_and_device_inputs():
    G = gpu_mod()
    import torch
    og, ctx = _pair()
    rng = np.random.default_rng(2)
    P, loc, U, f, y = G.mlp_samples(ctx, 9, 0, 130, device=True)   # one block + 2
    fh, yh = f.cpu().numpy(), y.cpu().numpy()
    nm = _norm_of(fh, yh)
    th = _rand_theta(rng)
    lg, gg = G.mlp_loss_grad(ctx, th, nm, f, y)
    assert isinstance(gg, torch.Tensor) and gg.is_cuda
    lo, go = O.mlp_loss_grad(th, nm, fh, yh)
    assert lg == pytest.approx(lo, rel=1e-6)
    assert np.linalg.norm(gg.cpu().numpy() - go) / np.linalg.norm(go) < 1e-5
    l1, g1 = G.mlp_loss_grad(ctx, th, nm, fh[:, :1].copy(), yh[:1].copy())
    o1, h1 = O.mlp_loss_grad(th, nm, fh[:, :1], yh[:1])
    assert l1 == pytest.approx(o1, rel=1e-6)
    assert np.linalg.norm(g1 - h1) / np.linalg.norm(h1) < 1e-5


def test_adamw_steps_match_oracle():
    G = gpu_mod()
    og, ctx = _pair()
    rng = np.random.default_rng(3)
    _, _, _, f, y = G.mlp_samples(ctx, 11, 0, 1000)
    nm = _norm_of(f, y)
    th0 = _rand_theta(rng, 0.2)
    lr, nsteps, batch = 1e-3, 5, 300        # 1500 samples: the set wraps once
    tg, lg = G.mlp_train_steps(ctx, th0, nm, f, y, batch, nsteps, lr, weight_decay=0.01)
    to, lo = O.mlp_train_steps(th0, nm, f, y, batch, nsteps, lr, wd=0.01)
    assert lg == pytest.approx(lo, rel=1e-5)
    # Adam normalises each gradient entry, so an FP32 gradient error shows up
    # as a fraction of lr per step; a wrong update rule moves entries by O(lr)
    d = (tg.astype(np.float64) - to.astype(np.float64))
    assert np.linalg.norm(d) / (lr * nsteps * np.sqrt(O.MLP_NPARAM)) < 2e-3
    assert np.abs(d).max() < 0.5 * lr * nsteps
    moved = np.linalg.norm(tg.astype(np.float64) - th0) / (lr * nsteps * np.sqrt(O.MLP_NPARAM))
    assert moved > 0.3


def test_bad_arguments_are_rejected():
    G = gpu_mod()
    og, ctx = _pair()
    U = np.zeros((9, 4))
    loc = np.zeros(4, dtype=np.int32)
    P = np.zeros((8, 4))
    with pytest.raises(G.GrmhdError):
        G.con2prim(ctx, U, loc, P, use_learned_guess=True)     # nothing loaded
    with pytest.raises(G.GrmhdError):
        G.mlp_get(ctx)
    th = np.zeros(O.MLP_NPARAM, dtype=np.float32)
    nm = np.ones(12, dtype=np.float32)
    nm[7] = 0.0
    with pytest.raises(G.GrmhdError):
        G.mlp_load(ctx, th, nm)                                  # zero std
    nm[7] = 1.0
    th[10] = np.nan
    with pytest.raises(G.GrmhdError):
        G.mlp_load(ctx, th, nm)


def _cold_guess(G, og, U, loc):
    """A start that knows nothing of the flow: rho = D, u from the energy
    above rest mass, no velocity, the field of U."""
    tab = og.geom_table(0)
    n2 = og.p.n2
    i, j = loc // n2, loc % n2
    gdet = tab[i + O.NG, j + O.NG, 32]
    alpha = tab[i + O.NG, j + O.NG, 33]
    D = alpha * U[0] / gdet
    P = np.zeros((8, U.shape[1]))
    P[0] = D
    P[1] = np.maximum(1e-3 * D, 0.1 * np.abs(U[1] / gdet * alpha + D))
    P[5:8] = U[5:8] / gdet
    return P


def test_trained_guess_keeps_the_root_and_cuts_newton_steps():
    G = gpu_mod()
    og, ctx = _pair(48, 64)
    rep = G.mlp_train(ctx, n_samples=1_000_000, n_val=50_000, seed=7, init_seed=1, epochs=3, batch=4096,
                      lr=3e-3, lr_min=3e-5, weight_decay=1e-4)
    assert rep["steps"] == (3 * 1_000_000 + 4095) // 4096
    assert rep["loss_last"] < 0.05 * rep["loss_first"]
    # a short run (3 epochs of 1e6 samples): log(W/D) to about 0.15, that is
    # W within ~15 %; longer runs on 1e7 samples reach about 0.05
    assert rep["val_rmse"] < 0.25
    # held-out states, far from the training indices
    P, loc, U, f, y = G.mlp_samples(ctx, 7, 5_000_000, 20000)
    g0 = _cold_guess(G, og, U, loc)
    Pp, fp, ip = G.con2prim(ctx, U, loc, g0.copy())
    Pl, fl, il = G.con2prim(ctx, U, loc, g0.copy(), use_learned_guess=True)
    # the oracle, started from the same learned W (GPU forward of the same
    # FP32 features), takes the same path
    th, nm = G.mlp_get(ctx)
    tab = og.geom_table(0)
    i, j = loc // og.p.n2, loc % og.p.n2
    D = tab[i + O.NG, j + O.NG, 33] * U[0] / tab[i + O.NG, j + O.NG, 32]
    wg = D * np.exp(G.mlp_forward(ctx, f).astype(np.float64))
    Po, fo, io = og.con2prim_w(U, loc, g0.copy(), wg)
    assert (fl == fo).mean() > 0.999
    # Newton's answer carries rounding times the conditioning of the
    # inversion (u recovered from W (1 - v^2) - D sqrt(1 - v^2)), as for the
    # plain inversion's parity: eps W (1 + sigma)/u for u, eps Gamma^2 (1 + sigma) for rho
    xi = np.array([[O.uniform(7, 16 * (5_000_000 + a) + k) for k in (4, 5)] for a in range(U.shape[1])])
    lor, sig = 50.0 ** xi[:, 0], 1e-3 * 1e5 ** xi[:, 1]
    eps = 2.220446049250313e-16
    cu = eps * lor ** 2 * (P[0] + GAM * P[1]) * (1 + sig) / P[1]
    cr = eps * lor ** 2 * (1 + sig)

    def close(Pa, Pb, mask):
        return ((np.abs(Pa[1] - Pb[1]) / Pb[1] / cu)[mask].max() < 4e3 and
                (np.abs(Pa[0] - Pb[0]) / Pb[0] / cr)[mask].max() < 4e3 and
                np.median(np.abs(Pa[1] - Pb[1]) / Pb[1]) < 1e-12)

    same = ((fl & O.C2P_FAIL) == 0) & (fl == fo)
    assert close(Pl, Po, same)
    assert (np.abs(il - io) <= 1).mean() > 0.99
    # same method, same root as the plain start where both converge by Newton
    both = (fp == O.C2P_NR) & (fl == O.C2P_NR)
    assert both.mean() > 0.4
    assert close(Pl, Pp, both)
    assert il[both].mean() < ip[both].mean()
    # the learned start leaves Newton no more often than the cold one
    assert (fl != O.C2P_NR).sum() <= (fp != O.C2P_NR).sum()


def _trained(ctx, samples=1_000_000, epochs=3):
    G = gpu_mod()
    rep = G.mlp_train(ctx, n_samples=samples, n_val=20_000, seed=7, init_seed=1, epochs=epochs, batch=4096,
                      lr=3e-3, lr_min=3e-5, weight_decay=1e-4)
    assert rep["val_rmse"] < 0.3
    return rep


def test_step_with_learned_rescue_matches_plain_start():
    """In the step the network is a rescue, tried only where Newton from the
    stage's own start does not converge: on a smooth torus that never
    happens, and the step is the plain step bit for bit."""
    G = gpu_mod()
    og, ctx = make_pair(64, 64, 1, gam=GAM)
    G.init_torus(ctx, beta0=100.0, pert_amp=0.04, seed=1)
    P0, U0, t0, dt0 = G.get_state(ctx)
    _trained(ctx)
    G.step(ctx, 5)
    Pa, Ua, ta, _ = G.get_state(ctx)
    da = G.diagnostics(ctx)
    G.set_state(ctx, P0, U0, t0, dt0)
    G.set_learned_guess(ctx, True)
    G.step(ctx, 5)
    Pb, Ub, tb, _ = G.get_state(ctx)
    db = G.diagnostics(ctx)
    G.set_learned_guess(ctx, False)
    assert tb == ta
    assert np.array_equal(Pa, Pb) and np.array_equal(Ua, Ub)
    assert db["n_learned"] == 0
    assert db["nr_iters"] == 2 * da["nr_iters"]


def _cold_restart(og, U):
    """Primitives a restart from conserved variables alone would start from:
    rho = D, u from the energy above rest mass, no velocity, the field of U."""
    n1, n2 = og.shape[0], og.shape[1]
    tab = og.geom_table(0)[O.NG:-O.NG, O.NG:-O.NG]
    gdet = tab[..., 32][..., None]
    alpha = tab[..., 33][..., None]
    D = alpha * U[0] / gdet
    P = np.zeros((8,) + U.shape[1:])
    P[0] = D
    P[1] = np.maximum(1e-3 * D, 0.1 * np.abs(U[1] / gdet * alpha + D))
    P[5:8] = U[5:8] / gdet
    return P


def test_learned_rescue_replaces_brent_in_the_step():
    """Zone class: zones whose stage primitives are a poor Newton start.  A
    64 x 64 x 1 grid is filled with held-out states of the training
    distribution (Lorentz factors up to 50, b^2/rho up to 100) whose
    primitives are replaced by a cold start (rho = D, no velocity), with
    Newton capped at 8 steps.  Without the network the zones that need more
    Newton steps from that start fall to the 1D Brent solve; with it, Newton
    from the network's W converges most of them: fewer Brent solves, and the
    same roots (the states after the step agree to the conditioning)."""
    G = gpu_mod()
    og, ctx = make_pair(64, 64, 1, gam=GAM, phys=dict(nr_maxit=8))
    _trained(ctx)
    n1, n2 = 64, 64
    # one held-out sample per zone, drawn at that zone's metric
    P, loc, U, f, y = G.mlp_samples(ctx, 7, 6_000_000, 40 * n1 * n2)
    pick = np.full(n1 * n2, -1)
    for a in range(loc.size):
        if pick[loc[a]] < 0:
            pick[loc[a]] = a
    assert (pick >= 0).all()
    Ug = np.ascontiguousarray(U[:, pick]).reshape(9, n1, n2, 1)
    Pc = np.ascontiguousarray(_cold_guess(G, og, U[:, pick], np.arange(n1 * n2))).reshape(8, n1, n2, 1)
    G.set_state(ctx, Pc, Ug, 0.0, 1e-12)
    d0 = G.diagnostics(ctx)
    G.step(ctx, 1)
    Pa, Ua = G.get_state(ctx)[:2]
    da = G.diagnostics(ctx)
    G.set_learned_guess(ctx, True)
    G.set_state(ctx, Pc, Ug, 0.0, 1e-12)
    G.step(ctx, 1)
    Pb, Ub = G.get_state(ctx)[:2]
    db = G.diagnostics(ctx)
    G.set_learned_guess(ctx, False)
    brent_plain = da["n_brent"] - d0["n_brent"]
    brent_learn = db["n_brent"] - da["n_brent"]
    learned = db["n_learned"] - da["n_learned"]
    print("cold starts in the step: Brent plain", brent_plain, "Brent with rescue", brent_learn, "rescued", learned,
          "Newton steps plain", da["nr_iters"] - d0["nr_iters"], "rescue", db["nr_iters"] - da["nr_iters"])
    assert brent_plain > 500
    assert learned > 0.5 * brent_plain
    assert brent_learn < 0.5 * brent_plain
    # the predictor's zones end at the same roots either way (to the
    # inversion's conditioning, up to eps Gamma^2 (1 + sigma) rho / u for u),
    # so the corrector starts from the same state
    for f in (0, 1):
        rel = np.abs(Pb[f] - Pa[f]) / np.abs(Pa[f])
        assert np.median(rel) < 1e-12 and rel.max() < 1e-3, (f, np.median(rel), rel.max())


def test_learned_rescue_zone_by_zone_work():
    """The stand-alone inversion in the step's order (use_learned_guess = 2)
    on held-out states from cold starts, Newton capped at 8 steps: every
    zone the network rescues ends at the root the plain order reaches through
    Brent, and the oracle's operation count of that zone's inversion is
    smaller along the learned path."""
    G = gpu_mod()
    og, ctx = make_pair(48, 64, 1, gam=GAM, phys=dict(nr_maxit=8))
    _trained(ctx)
    P, loc, U, f, y = G.mlp_samples(ctx, 7, 5_000_000, 4000)
    g0 = _cold_guess(G, og, U, loc)
    Pp, fp, ip = G.con2prim(ctx, U, loc, g0.copy())
    Pr, fr, ir = G.con2prim(ctx, U, loc, g0.copy(), use_learned_guess=2)
    rescued = (fr & G.C2P_LEARNED) != 0
    assert rescued.sum() > 100
    # a rescued zone is one whose plain Newton did not converge
    assert np.all(fp[rescued] != G.C2P_NR)
    brent = rescued & (fp == G.C2P_BRENT_W)
    assert brent.sum() > 50
    rel = np.abs(Pr[:2, brent] - Pp[:2, brent]) / np.abs(Pp[:2, brent])
    assert np.median(rel) < 1e-12 and rel.max() < 1e-6
    th, nm = G.mlp_get(ctx)
    tab = og.geom_table(0)
    i, j = loc // og.p.n2, loc % og.p.n2
    D = tab[i + O.NG, j + O.NG, 33] * U[0] / tab[i + O.NG, j + O.NG, 32]
    wl = D * np.exp(G.mlp_forward(ctx, f).astype(np.float64))
    # per zone: plain = set-up + Newton from the guess (fails) + Brent;
    # rescue = set-up + Newton from the guess (fails) + Newton from the
    # network's W, counted as plain - (set-up + Brent) + (set-up + learned Newton)
    plain_flops = rescue_flops = brent_part = learned_part = 0
    for a in np.flatnonzero(brent)[:200]:
        geom = tab[i[a] + O.NG, j[a] + O.NG]
        kw = dict(nr_maxit=8)
        A = O.count_con2prim(U[:, a], geom, g0[:, a], GAM, methods=15, **kw)[3]["flops"]
        B = O.count_con2prim(U[:, a], geom, g0[:, a], GAM, methods=10, **kw)[3]["flops"]
        Cc = O.count_con2prim(U[:, a], geom, g0[:, a], GAM, methods=15, wguess=wl[a], **kw)[3]["flops"]
        plain_flops += A
        rescue_flops += A - B + Cc
        brent_part += B
        learned_part += Cc
    print("rescued Brent zones: oracle flops plain", plain_flops, "rescue", rescue_flops,
          "Brent (with set-up)", brent_part, "Newton from the network's W (with set-up)", learned_part)
    assert learned_part < brent_part
    assert rescue_flops < 0.9 * plain_flops


