"""The polar cylindrification (Section 4.1; the band reading of the grid
parameters cyl_r, cyl_dx2) on the GPU against the oracle's: the centre
metric through prim2cons, the face metric through the fluxes and the CFL
step, the connection through whole steps (FP64 path: 1e-10 per field, the
metric of gpu_common.field_err), the torus set-up, a ragged 3D grid, PPM
faces, the mixed path (1e-4 per step on every zone) and the refusals."""
import numpy as np
import pytest

import oracle
from tests import inputs
from tests.gpu_common import field_err, gpu_mod, make_pair

pytestmark = pytest.mark.gpu
TOL = 1e-10
CYL = dict(cyl_r=2.2, cyl_dx2=0.25)


def _torus(n1=64, n2=64, n3=1, precision=0, **kw):
    og, ctx = make_pair(n1, n2, n3, gam=13.0 / 9.0, precision=precision, **CYL, **kw)
    og.init_torus(pert_amp=0.04, seed=1)
    return og, ctx


def test_cyl_prim2cons_in_the_bands():
    G = gpu_mod()
    n1, n2 = 40, 36
    og, ctx = make_pair(n1, n2, 1, gam=4.0 / 3.0, r_out=1000.0, cyl_r=1.8, cyl_dx2=0.3)
    tab = og.geom_table(0)
    loc = inputs.zone_locations(4000, n1, n2, 5, i_h=og.i_h)
    i, j = loc // n2, loc % n2
    gsp = tab[i + oracle.NG, j + oracle.NG, :16].reshape(-1, 4, 4)[:, 1:, 1:]
    P = inputs.place_prims(inputs.prim_params(loc.size, 6), gsp)
    Uo = og.prim2cons(P, loc)
    Ug = G.prim2cons(ctx, P, loc)
    for c in range(9):
        s = np.abs(Uo[c]).max()
        assert np.abs(Ug[c] - Uo[c]).max() <= 1e-13 * s, c


def test_cyl_torus_init_fluxes_and_dt():
    G = gpu_mod()
    og, ctx = _torus()
    G.init_torus(ctx, pert_amp=0.04, seed=1)
    Pg, Ug, tg, dtg = G.get_state(ctx)
    Po, Uo, to, dto = og.get_state()
    assert field_err(Pg, Po).max() < 1e-9
    assert field_err(Ug, Uo).max() < 1e-9
    assert dtg == pytest.approx(dto, rel=1e-12)
    G.set_state(ctx, Po, Uo, to, dto)
    Fo, dt_o = og.fluxes()
    Fg, dt_g = G.fluxes(ctx)
    assert dt_g == pytest.approx(dt_o, rel=1e-13)
    for d in range(3):
        for c in range(9):
            s = np.abs(Fo[d, c]).max() + np.abs(Uo[c]).max()
            assert np.abs(Fg[d, c] - Fo[d, c]).max() <= 1e-13 * s, (d, c)
    # in the rows of the lower band (X2 width 0.25 = 8 rows) the cylindrified
    # fluxes are not the MKS ones
    ref, _ = make_pair(64, 64, 1, gam=13.0 / 9.0)
    ref.set_state(Po, Uo, to, dto)
    band = np.s_[:, :, :, :8]
    assert np.abs(ref.fluxes()[0][band] - Fo[band]).max() > 1e-3 * np.abs(Fo[band]).max()


def test_cyl_steps_per_step_parity():
    G = gpu_mod()
    og, ctx = _torus()
    worst = 0.0
    for _ in range(10):
        Po, Uo, to, dto = og.get_state()
        G.set_state(ctx, Po, Uo, to, dto)
        og.step()
        G.step(ctx)
        e = max(field_err(G.get_state(ctx)[0], og.get_state()[0]).max(),
                field_err(G.get_state(ctx)[1], og.get_state()[1]).max())
        worst = max(worst, e)
    assert worst < TOL, worst
    do, dg = og.diagnostics(), G.diagnostics(ctx)
    for k in ("n_nr", "n_brent", "n_entropy", "n_entropy_beta", "n_fail", "n_ceil", "n_gcap", "n_fixed"):
        assert dg[k] == do[k], k
    assert dg["divb_max"] < 1e-11


@pytest.mark.parametrize("recon", [oracle.PLM, oracle.PPM])
def test_cyl_3d_ragged_grid(recon):
    G = gpu_mod()
    og, ctx = make_pair(19, 14, 6, gam=4.0 / 3.0, r_out=30.0, cyl_r=1.8, cyl_dx2=0.3, recon=recon)
    og.init_torus(pert_amp=0.02, seed=2)
    G.init_torus(ctx, pert_amp=0.02, seed=2)
    assert field_err(G.get_state(ctx)[0], og.get_state()[0]).max() < 1e-9
    for _ in range(3):
        Po, Uo, to, dto = og.get_state()
        G.set_state(ctx, Po, Uo, to, dto)
        og.step()
        G.step(ctx)
        eP = field_err(G.get_state(ctx)[0], og.get_state()[0])
        eU = field_err(G.get_state(ctx)[1], og.get_state()[1])
        assert max(eP.max(), eU.max()) < TOL, (eP, eU)


def test_cyl_mixed_one_step_every_zone():
    G = gpu_mod()
    og, ctx = make_pair(48, 48, 8, gam=4.0 / 3.0, r_out=1000.0, precision=1, cyl_r=1.6, cyl_dx2=0.25)
    og.init_torus(r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.02, seed=2)
    Po, Uo, to, dto = og.get_state()
    G.set_state(ctx, Po, Uo, to, dto)
    og.step()
    G.step(ctx)
    eP = field_err(G.get_state(ctx)[0], og.get_state()[0])
    eU = field_err(G.get_state(ctx)[1], og.get_state()[1])
    print("cylindrified mixed one step: P", eP, "U", eU)
    assert eP.max() < 1e-4, eP
    assert eU[:8].max() < 1e-5, eU


@pytest.mark.parametrize("kw", [dict(cyl_r=5.0, cyl_dx2=0.25), dict(cyl_r=2.0, cyl_dx2=0.0),
                                dict(cyl_r=2.0, cyl_dx2=1.5)])
def test_cyl_refusals(kw):
    G = gpu_mod()
    gp = G.default_grid(32, 32, 1, **kw)
    ctx = G.init_grid(gp, G.default_phys())
    with pytest.raises(G.GrmhdError):
        G.set_metric(ctx, 0.9375)


def test_cyl_refused_on_flat_space():
    G = gpu_mod()
    gp = G.default_grid(8, 8, 8, metric=G.MINK_CART, cyl_r=2.0, cyl_dx2=0.25)
    ctx = G.init_grid(gp, G.default_phys())
    with pytest.raises(G.GrmhdError):
        G.set_metric(ctx, 0.0, G.MINK_CART)
