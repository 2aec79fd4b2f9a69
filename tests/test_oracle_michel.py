"""The oracle's whole curved-space step (fluxes, connection sources, RK2,
inversion, radial boundaries) pinned by an exact steady solution: Michel
accretion onto a Schwarzschild black hole (a = 0, Kerr-Schild).  The steady
flow must be held with second-order convergence under refinement, its
construction must satisfy the two conservation laws it came from, and the
horizon mass flux must equal the analytic 4 pi r^2 rho u."""
import math

import numpy as np
import pytest

import oracle as O
from tests.michel import Michel, michel_prims

GAM = 4.0 / 3.0
N_POLY = 1.0 / (GAM - 1.0)


def _grid(n1, n2=8):
    p = O.default_params(n1=n1, n2=n2, n3=1, a=0.0, r_out=20.0, gam=GAM)
    return O.Grid(p)


def _loc(og):
    n1, n2, n3 = og.shape
    return np.repeat((np.arange(n1)[:, None] * n2 + np.arange(n2)[None, :]).reshape(-1), n3).astype(np.int32)


def _start(og, mic):
    P = michel_prims(og, mic, GAM)
    U = og.prim2cons(P.reshape(8, -1), _loc(og)).reshape((9,) + og.shape)
    og.set_state(P, U, 0.0, 0.0)
    og.set_dt(og.initial_dt())
    return P


def test_michel_construction_is_consistent():
    mic = Michel(r_c=8.0, n=N_POLY)
    for r in (2.2, 4.0, 8.0, 12.0, 19.0):
        rho, T, u = mic.state(r)
        h = 1.0 + (N_POLY + 1.0) * T
        assert r * r * rho * u == pytest.approx(mic.mdot, rel=1e-12)
        assert h * h * (1.0 - 2.0 / r + u * u) == pytest.approx(mic.bern, rel=1e-12)
        a2 = (N_POLY + 1.0) * T / (N_POLY * h)
        # the coordinate speed of sound relative to the flow, u^2 / (1 - 2/r + u^2),
        # is below a^2 outside the sonic radius and above it inside
        v2 = u * u / (1.0 - 2.0 / r + u * u)
        if r > 8.0:
            assert v2 < a2
        elif r < 8.0:
            assert v2 > a2
    # the primitives satisfy u.u = -1 with u^r of the solution
    og = _grid(32)
    P = michel_prims(og, mic, GAM)
    tab = og.geom_table(0)
    for i in (0, 5, 17, 31):
        g = O.geom_from(tab[i + O.NG, 4 + O.NG, :16].reshape(4, 4))
        s, _ = O.state_of(P[:, i, 4, 0], g)
        r = og.r_of_x1(og.x1in + (i + 0.5) * og.dx[0])
        assert s["ucon"][1] * r == pytest.approx(-mic.state(r)[2], rel=1e-12)
        assert s["ucon"] @ s["ucov"] == pytest.approx(-1.0, abs=1e-12)


def _drift(n1, n2, t_end=4.0):
    mic = Michel(r_c=8.0, n=N_POLY)
    og = _grid(n1, n2)
    P0 = _start(og, mic)
    while True:
        _, _, t, dt = og.get_state()
        if t >= t_end - 1e-12:
            break
        if t + dt > t_end:
            og.set_dt(t_end - t)
        assert og.step() == 0
    P = og.get_state()[0]
    r = np.array([og.r_of_x1(og.x1in + (i + 0.5) * og.dx[0]) for i in range(n1)])
    # away from the outer boundary, whose inflow reset travels in at c_s + u
    band = (r > 3.0) & (r < 12.0)
    return np.abs(P[0, band, :, 0] / P0[0, band, :, 0] - 1.0).mean(), og


def test_michel_flow_is_held_at_second_order():
    # both directions refined: the discrete balance of the theta pressure flux
    # against the connection source is second order in the theta spacing
    e = [_drift(n1, n2)[0] for n1, n2 in ((32, 8), (64, 16), (128, 32))]
    assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0, e
    assert e[2] < 1e-3


def _horizon_mdot_error(n2):
    mic = Michel(r_c=8.0, n=N_POLY)
    og = _grid(16, n2)
    _start(og, mic)
    d = og.diagnostics()
    # Eq. 38 at the first zone with r >= r_H, sum sqrt(-g) rho u^1 dX2 dX3, is
    # the midpoint rule for the integral over the sphere, 4 pi r^2 rho u^r
    i = og.i_h
    r = og.r_of_x1(og.x1in + (i + 0.5) * og.dx[0])
    rho, T, u = mic.state(r)
    return d["mdot"] / (-4.0 * math.pi * r * r * rho * u) - 1.0


def test_michel_horizon_mass_flux():
    e = [abs(_horizon_mdot_error(n2)) for n2 in (16, 32, 64)]
    assert e[0] / e[1] > 3.5 and e[1] / e[2] > 3.5, e
    assert e[2] < 2e-3


def test_michel_horizon_efficiency():
    """(Edot - Mdot)/|Mdot| of Eqs. 38 and 41: for the radial flow without
    field every zone of the shell has T^r_t = rho h u^r u_t with the same
    h u_t, so Edot = -h u_t Mdot and the ratio is 1 + h u_t = 1 - sqrt(B),
    B = h^2 (1 - 2/r + u^2) the Bernoulli constant (u_t is the same in
    Schwarzschild and Kerr-Schild time) -- at any resolution."""
    mic = Michel(r_c=8.0, n=N_POLY)
    og = _grid(16, 12)
    _start(og, mic)
    d = og.diagnostics()
    assert d["mdot"] < 0.0 and d["edot"] < 0.0
    assert d["eta"] == pytest.approx(1.0 - math.sqrt(mic.bern), abs=1e-12)
    assert d["eta"] == pytest.approx((d["edot"] - d["mdot"]) / abs(d["mdot"]), rel=1e-15)
