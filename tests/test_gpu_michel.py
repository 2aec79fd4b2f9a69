"""GPU (C ABI) against the oracle on Michel accretion onto a Schwarzschild
black hole (a = 0): one step from the same state and a free-running window in
FP64, and the mixed path holding the steady flow as well as the FP64 path."""
import numpy as np

import oracle as O
from tests.gpu_common import field_err, gpu_mod, make_pair
from tests.michel import Michel, michel_prims

import pytest

pytestmark = pytest.mark.gpu
GAM = 4.0 / 3.0


def _michel_pair(n1, n2, precision=0):
    og, ctx = make_pair(n1, n2, 1, gam=GAM, a=0.0, r_out=20.0, precision=precision)
    n = n1 * n2
    loc = np.repeat(np.arange(n, dtype=np.int32), 1)
    P = michel_prims(og, Michel(r_c=8.0, n=1.0 / (GAM - 1.0)), GAM)
    U = og.prim2cons(P.reshape(8, -1), loc).reshape((9,) + og.shape)
    og.set_state(P, U, 0.0, 0.0)
    dt = og.initial_dt()
    og.set_dt(dt)
    return og, ctx, P, U, dt


def test_michel_one_step_parity():
    G = gpu_mod()
    og, ctx, P, U, dt = _michel_pair(72, 20)
    G.set_state(ctx, P, U, 0.0, dt)
    og.step()
    G.step(ctx, 1)
    Po, Uo, to, _ = og.get_state()
    Pg, Ug, tg, _ = G.get_state(ctx)
    assert tg == to
    assert field_err(Pg, Po).max() < 1e-10
    assert field_err(Ug, Uo).max() < 1e-10


def test_michel_free_running_parity():
    G = gpu_mod()
    og, ctx, P, U, dt = _michel_pair(40, 12)
    G.set_state(ctx, P, U, 0.0, dt)
    og.step(25)
    G.step(ctx, 25)
    Po, Uo, to, dto = og.get_state()
    Pg, Ug, tg, dtg = G.get_state(ctx)
    assert tg == pytest.approx(to, rel=1e-12) and dtg == pytest.approx(dto, rel=1e-10)
    assert field_err(Pg, Po).max() < 1e-8
    assert field_err(Ug, Uo).max() < 1e-8


def test_michel_mixed_holds_the_flow_like_fp64():
    G = gpu_mod()
    drift = {}
    for prec in (0, 1):
        og, ctx, P, U, dt = _michel_pair(96, 24, precision=prec)
        G.set_state(ctx, P, U, 0.0, dt)
        G.step(ctx, 60)
        Pg = G.get_state(ctx)[0]
        r = np.array([og.r_of_x1(og.x1in + (i + 0.5) * og.dx[0]) for i in range(96)])
        band = (r > 3.0) & (r < 12.0)
        drift[prec] = Pg[0, band] / P[0, band] - 1.0
    # the mixed path's deviation from the steady flow is the FP64 path's
    # truncation error plus FP32 rounding of the fluxes
    assert np.abs(drift[1] - drift[0]).max() < 1e-4
    assert np.abs(drift[0]).mean() < 1e-2
