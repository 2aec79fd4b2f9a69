"""GPU (C ABI) against the oracle on magnetised flat-space shock tubes, where
the MC limiter switches branches and the fluxes jump: one step from the same
state, a free-running window, and the hydrodynamic tube's convergence to the
exact Riemann solution holding for the GPU too (mixed path)."""
import math

import numpy as np
import pytest

import oracle
from tests.gpu_common import field_err, gpu_mod, make_pair
from tests.riemann import ExactRiemann, State

pytestmark = pytest.mark.gpu
GAM = 4.0 / 3.0
LEFT = State(5.0, 4.0, 0.2)
RIGHT = State(1.0, 0.1, -0.1)


def _tube_pair(n, precision=0):
    box = dict(x1min=0.0, x1max=1.0, x2min=0.0, x2max=1.0, x3min=0.0, x3max=1.0,
               bc1=oracle.BC_OUTFLOW, bc2=oracle.BC_OUTFLOW, bc3=oracle.BC_OUTFLOW)
    return make_pair(n, 1, 1, gam=GAM, metric=oracle.MINK_CART, precision=precision, **box)


def _prims(n, B=None):
    x = (np.arange(n) + 0.5) / n
    P = np.zeros((8, n, 1, 1))
    for st, sel, b in ((LEFT, x < 0.5, 0), (RIGHT, x >= 0.5, 1)):
        P[0, sel] = st.rho
        P[1, sel] = st.p / (GAM - 1.0)
        P[2, sel] = st.v / math.sqrt(1.0 - st.v ** 2)
        if B is not None:
            for c in range(3):
                P[5 + c, sel] = B[b][c]
    return x, P


def _start(og, ctx, P):
    G = gpu_mod()
    U = og.prim2cons(P.reshape(8, -1), np.zeros(P[0].size, dtype=np.int32)).reshape((9,) + P.shape[1:])
    og.set_state(P, U, 0.0, 0.0)
    dt = og.initial_dt()
    og.set_dt(dt)
    G.set_state(ctx, P, U, 0.0, dt)


B_TUBE = ((0.5, 1.0, 0.3), (0.5, -0.7, 0.2))


def test_magnetised_tube_one_step_and_window():
    G = gpu_mod()
    og, ctx = _tube_pair(203)          # 203 zones: 1 + 1/128 blocks of zones, ragged
    x, P = _prims(203, B_TUBE)
    _start(og, ctx, P)
    og.step()
    G.step(ctx, 1)
    assert field_err(G.get_state(ctx)[0], og.get_state()[0]).max() < 1e-10
    assert field_err(G.get_state(ctx)[1], og.get_state()[1]).max() < 1e-10
    og.step(40)
    G.step(ctx, 40)
    Po, Uo, to, _ = og.get_state()
    Pg, Ug, tg, _ = G.get_state(ctx)
    assert tg == pytest.approx(to, rel=1e-12)
    assert field_err(Pg, Po).max() < 1e-8
    assert field_err(Ug, Uo).max() < 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_hydro_tube_approaches_the_exact_solution(precision):
    G = gpu_mod()
    ex = ExactRiemann(LEFT, RIGHT, GAM)
    errs = []
    for n in (128, 256):
        og, ctx = _tube_pair(n, precision)
        x, P = _prims(n)
        _start(og, ctx, P)
        t_end = 0.3
        while True:
            t, dt = G.get_state(ctx)[2:]
            if t >= t_end - 1e-12:
                break
            if t + dt > t_end:
                Pg, Ug, t, _ = G.get_state(ctx)
                G.set_state(ctx, Pg, Ug, t, t_end - t)
            G.step(ctx, 1)
        rho = G.get_state(ctx)[0][0, :, 0, 0]
        rho_ex = np.array([ex.sample((xi - 0.5) / t_end)[0] for xi in x])
        errs.append(np.abs(rho - rho_ex).mean())
    assert errs[0] / errs[1] > 1.5, errs
    assert errs[1] < 0.06
