"""The PPM faces (GRMHD_PPM: the parabolic reconstruction Section 2.2 names
after its PLM) on the GPU against the oracle's PPM: face fluxes, single steps
from the same state (FP64 path: 1e-10 per field, the metric of
gpu_common.field_err), a ragged 3D grid, flat space with LLF and HLL, the
mixed path (1e-4 per step on every zone), and the refusal of a PPM member by
the batched ensemble."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import field_err, gpu_mod, make_pair

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _torus(n1=64, n2=64, n3=1, precision=0, **kw):
    og, ctx = make_pair(n1, n2, n3, gam=13.0 / 9.0, precision=precision, recon=oracle.PPM, **kw)
    og.init_torus(pert_amp=0.04, seed=1)
    return og, ctx


def test_ppm_face_fluxes():
    G = gpu_mod()
    og, ctx = _torus()
    Po, Uo, to, dto = og.get_state()
    G.set_state(ctx, Po, Uo, to, dto)
    Fo, dt_o = og.fluxes()
    Fg, dt_g = G.fluxes(ctx)
    assert dt_g == pytest.approx(dt_o, rel=1e-13)
    for d in range(3):
        for c in range(9):
            s = np.abs(Fo[d, c]).max() + np.abs(Uo[c]).max()
            assert np.abs(Fg[d, c] - Fo[d, c]).max() <= 1e-13 * s, (d, c)
    # the PPM fluxes are not the PLM ones
    og2, ctx2 = make_pair(64, 64, 1, gam=13.0 / 9.0)
    og2.set_state(Po, Uo, to, dto)
    assert np.abs(og2.fluxes()[0] - Fo).max() > 1e-6 * np.abs(Fo).max()


def test_ppm_steps_per_step_parity():
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


def test_ppm_3d_ragged_grid():
    G = gpu_mod()
    og, ctx = make_pair(19, 14, 6, gam=4.0 / 3.0, r_out=30.0, recon=oracle.PPM)
    og.init_torus(pert_amp=0.02, seed=2)
    G.init_torus(ctx, pert_amp=0.02, seed=2)
    for _ in range(3):
        Po, Uo, to, dto = og.get_state()
        G.set_state(ctx, Po, Uo, to, dto)
        og.step()
        G.step(ctx)
        eP = field_err(G.get_state(ctx)[0], og.get_state()[0])
        eU = field_err(G.get_state(ctx)[1], og.get_state()[1])
        assert max(eP.max(), eU.max()) < TOL, (eP, eU)


@pytest.mark.parametrize("riemann", [oracle.LLF, oracle.HLL])
def test_ppm_flat_space(riemann):
    G = gpu_mod()
    box = dict(x1min=0.0, x1max=1.0, x2min=0.0, x2max=1.0, x3min=0.0, x3max=1.0,
               bc1=oracle.BC_PERIODIC, bc2=oracle.BC_OUTFLOW, bc3=oracle.BC_PERIODIC, recon=oracle.PPM)
    n1, n2, n3 = 13, 11, 9
    og, ctx = make_pair(n1, n2, n3, gam=5.0 / 3.0, metric=oracle.MINK_CART, riemann=riemann, **box)
    x = (np.arange(n1) + 0.5) / n1
    y = (np.arange(n2) + 0.5) / n2
    z = (np.arange(n3) + 0.5) / n3
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    tp = 2 * np.pi
    P = np.zeros((8, n1, n2, n3))
    P[0] = 1.0 + 0.3 * np.sin(tp * X) * np.cos(tp * Y)
    P[1] = 0.6 + 0.2 * np.cos(tp * (X + Z))
    P[2] = 0.3 * np.sin(tp * Y)
    P[3] = -0.2 * np.cos(tp * Z)
    P[4] = 0.25 * np.sin(tp * (X - Y))
    P[5] = 0.2 + 0.1 * np.sin(tp * Y)
    P[6] = 0.1 * np.cos(tp * Z)
    P[7] = 0.15 * np.sin(tp * X)
    U = og.prim2cons(P.reshape(8, -1), np.zeros(n1 * n2 * n3, dtype=np.int32)).reshape((9, n1, n2, n3))
    og.set_state(P, U, 0.0, 0.0)
    dt = og.initial_dt()
    G.set_state(ctx, P, U, 0.0, dt)
    for _ in range(3):
        og.step()
        G.step(ctx)
    assert field_err(G.get_state(ctx)[0], og.get_state()[0]).max() < 1e-9


def test_ppm_mixed_one_step_every_zone():
    G = gpu_mod()
    og, ctx = make_pair(48, 48, 8, gam=4.0 / 3.0, r_out=1000.0, precision=1, recon=oracle.PPM)
    og.init_torus(r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.02, seed=2)
    Po, Uo, to, dto = og.get_state()
    G.set_state(ctx, Po, Uo, to, dto)
    og.step()
    G.step(ctx)
    eP = field_err(G.get_state(ctx)[0], og.get_state()[0])
    eU = field_err(G.get_state(ctx)[1], og.get_state()[1])
    print("PPM mixed one step: P", eP, "U", eU)
    assert eP.max() < 1e-4, eP
    assert eU[:8].max() < 1e-5, eU


def test_ensemble_refuses_a_ppm_member():
    G = gpu_mod()
    _, a = make_pair(16, 16, 1, gam=13.0 / 9.0)
    _, b = _torus(16, 16)
    G.init_torus(a, pert_amp=0.0)
    G.init_torus(b, pert_amp=0.0)
    with pytest.raises(G.GrmhdError):
        G.ensemble_create([a, b])


@pytest.mark.parametrize("precision", [0, 1])
def test_ppm_columns_and_row_warps_96cubed(precision):
    """At 96^3 the X1 / X2 sweeps walk columns of 4 faces and the X3 sweep
    runs one warp per row (both paths): face fluxes and one step against the
    oracle (FP64: 1e-13 of the LLF scale per face, 1e-10 per field after
    the step, u of the cold atmosphere at r_out = 1000 M measured against
    rho + u, the precision its inversion from E - D gives it; mixed: the
    FP32 face scale and 1e-4 on every zone)."""
    G = gpu_mod()
    og, ctx = make_pair(96, 96, 96, gam=4.0 / 3.0, r_out=1000.0, precision=precision, recon=oracle.PPM)
    og.init_torus(pert_amp=0.02, seed=2)
    Po, Uo, to, dto = og.get_state()
    G.set_state(ctx, Po, Uo, to, dto)
    Fo, dt_o = og.fluxes()
    Fg, dt_g = G.fluxes(ctx)
    ftol = 1e-13 if precision == 0 else 2e-6
    if precision == 1:
        Fo[:, 1] += Fo[:, 0]  # the mixed path carries the energy flux rest-mass subtracted
    assert dt_g == pytest.approx(dt_o, rel=1e-13 if precision == 0 else 1e-5)
    for d in range(3):
        for c in range(9):
            s = np.abs(Fo[d, c]).max() + np.abs(Uo[c]).max()
            assert np.abs(Fg[d, c] - Fo[d, c]).max() <= ftol * s, (d, c)
    og.step()
    G.step(ctx)
    Pg, Ug = G.get_state(ctx)[:2]
    P1, U1 = og.get_state()[:2]
    eP, eU = field_err(Pg, P1), field_err(Ug, U1)
    if precision == 0:
        assert max(np.delete(eP, 1).max(), eU.max()) < TOL, (eP, eU)
        assert (np.abs(Pg[1] - P1[1]) / (P1[0] + P1[1])).max() < TOL
    else:
        assert eP.max() < 1e-4 and eU[:8].max() < 1e-5, (eP, eU)
