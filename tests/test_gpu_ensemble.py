"""Ensemble of independent tori stepped by persistent launches over a ragged
tile list (members above a size threshold on their own kernels, on parallel
branches of the same graph): every member must evolve bit-for-bit as the same torus alone, for any
tiling and threshold, and the autotuner must leave the members' state
untouched."""
import numpy as np
import pytest

from tests.gpu_common import gpu_mod

pytestmark = pytest.mark.gpu

MEMBERS = [  # (n1, n2, n3, spin, gamma, beta0, seed)
    (40, 32, 1, 0.9375, 13.0 / 9.0, 100.0, 11),
    (24, 20, 6, 0.5, 4.0 / 3.0, 50.0, 12),
    (33, 17, 1, 0.0, 5.0 / 3.0, 300.0, 13),
    (20, 24, 9, 0.98, 4.0 / 3.0, 30.0, 14),
    (48, 40, 1, 0.7, 13.0 / 9.0, 150.0, 15),
]


def _member(G, torch, spec, precision, **kw):
    n1, n2, n3, a, gam, b0, seed = spec
    gp = G.default_grid(n1, n2, n3, a=a, r_out=60.0, precision=precision, **kw)
    gp.stream = torch.cuda.current_stream().cuda_stream
    ctx = G.init_grid(gp, G.default_phys(gam=gam))
    G.set_metric(ctx, a, G.KERR_MKS)
    G.init_torus(ctx, r_in=6.0, r_max=12.0, beta0=b0, pert_amp=0.04, seed=seed)
    return ctx


@pytest.mark.parametrize("precision", [0, 1])
def test_members_evolve_as_alone(precision):
    torch = pytest.importorskip("torch")
    G = gpu_mod()
    ens_members = [_member(G, torch, s, precision) for s in MEMBERS]
    solo = [_member(G, torch, s, precision) for s in MEMBERS]
    ens = G.ensemble_create(ens_members)
    G.ensemble_step(ens, 2)
    G.ensemble_set_tiling(ens, 1, 4, 16, 2)   # a different tiling mid-run
    G.ensemble_step(ens, 2)
    # members of >= 2^12 zones on their own kernels inside the graph, the rest batched
    G.ensemble_set_tiling(ens, 2, 2, 8, 3, solo_log2=12)
    G.ensemble_step(ens, 2)
    # four members on parallel branches of the graph, one batched beside them
    G.ensemble_set_tiling(ens, 2, 2, 8, 3, solo_log2=10)
    G.ensemble_step(ens, 2)
    G.ensemble_sync(ens)
    for c in solo:
        G.step(c, 8)
    for a, b in zip(ens_members, solo):
        Pa, Ua, ta, dta = G.get_state(a)
        Pb, Ub, tb, dtb = G.get_state(b)
        assert np.array_equal(Pa, Pb) and np.array_equal(Ua, Ub)
        assert ta == tb and dta == dtb
        da, db = G.diagnostics(a), G.diagnostics(b)
        for k in ("n_nr", "nr_iters", "n_floor", "n_fail", "n_steps"):
            assert da[k] == db[k], k
    ens.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_cylindrified_and_hll_members_evolve_as_alone(precision):
    """Members with the polar cylindrification (their band rows' metric) and
    one with the HLL flux, batched beside plain ones, step bit for bit as
    alone."""
    torch = pytest.importorskip("torch")
    G = gpu_mod()
    kws = [dict(cyl_r=1.8, cyl_dx2=0.3), dict(riemann=G.HLL), dict(cyl_r=1.6, cyl_dx2=0.25, riemann=G.HLL), {}]
    specs = MEMBERS[:4]
    mem = [_member(G, torch, s, precision, **k) for s, k in zip(specs, kws)]
    solo = [_member(G, torch, s, precision, **k) for s, k in zip(specs, kws)]
    ens = G.ensemble_create(mem)
    G.ensemble_step(ens, 3)
    G.ensemble_sync(ens)
    for c in solo:
        G.step(c, 3)
    for a, b in zip(mem, solo):
        Pa, Ua, ta, dta = G.get_state(a)
        Pb, Ub, tb, dtb = G.get_state(b)
        assert np.array_equal(Pa, Pb) and np.array_equal(Ua, Ub)
        assert ta == tb and dta == dtb
    ens.close()


def test_autotune_restores_state_and_keeps_results():
    torch = pytest.importorskip("torch")
    G = gpu_mod()
    mem = [_member(G, torch, s, 1) for s in MEMBERS]
    solo = [_member(G, torch, s, 1) for s in MEMBERS]
    ens = G.ensemble_create(mem)
    G.ensemble_step(ens, 1)
    before = [G.get_state(c) for c in mem]
    cnt_before = [G.diagnostics(c)["n_steps"] for c in mem]
    tiling, ms = G.ensemble_autotune(ens, 1)
    assert ms > 0 and 1 <= tiling["items_flux"] <= 16
    assert tiling["solo_log2"] == 0 or 10 <= tiling["solo_log2"] <= 40
    for c, b, n in zip(mem, before, cnt_before):
        P, U, t, dt = G.get_state(c)
        assert np.array_equal(P, b[0]) and np.array_equal(U, b[1]) and t == b[2] and dt == b[3]
        assert G.diagnostics(c)["n_steps"] == n
    G.ensemble_step(ens, 2)
    G.ensemble_sync(ens)
    for c in solo:
        G.step(c, 3)
    for a, b in zip(mem, solo):
        assert np.array_equal(G.get_state(a)[0], G.get_state(b)[0])
    assert G.ensemble_get_tiling(ens) == tiling
    ens.close()
