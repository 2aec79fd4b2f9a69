"""The oracle's horizon angular-momentum flux (Eq. 40) pinned by a closed form.

On a Schwarzschild black hole (a = 0) in Kerr-Schild coordinates, take a
uniform, unmagnetised fluid whose modified velocity is purely azimuthal with
ut^3 = v0 / (r sin theta).  Then Gamma = sqrt(1 + v0^2) is uniform, u_phi =
g_phiphi u^phi = r sin theta v0, and, with ut^r = 0, u^r = -Gamma alpha g^{tr}
= -2 Gamma alpha / r (g^{tr} = 2/r, alpha = 1/sqrt(1 + 2/r)).  The flux
through the sphere of radius r,

  Ldot = int int sqrt(-g) T^r_phi dtheta dphi
       = int int r^2 sin theta (rho + u + p) u^r u_phi dtheta dphi
       = -2 pi^2 (rho + u + p) Gamma alpha v0 r^2,

is the limit of the midpoint sums over the horizon zones.  In the code
coordinate X2 the integrand sin^2 theta(X2) dtheta/dX2 is smooth and
periodic (theta(X2 + 2) = theta(X2) + pi), and midpoint sums of a smooth
periodic function converge faster than any power of dX2, so already 16 rows
reproduce the closed form to round-off.  A wrong component (T^1_2, T^3_1), a
missing sqrt(-g) or Jacobian, or a flipped sign fails the comparison.
"""
import math

import numpy as np
import pytest

import oracle as O

GAM = 4.0 / 3.0
RHO, UU, V0 = 0.3, 0.05, 0.4


def _grid(n2):
    og = O.Grid(O.default_params(n1=24, n2=n2, n3=1, a=0.0, r_out=20.0, gam=GAM))
    n1 = og.shape[0]
    tab = og.geom_table(0)
    P = np.zeros((8, n1, n2, 1))
    P[0], P[1] = RHO, UU
    for i in range(n1):
        for j in range(n2):
            gphph = tab[i + O.NG, j + O.NG, 15]           # g_33 = r^2 sin^2 theta (dphi/dX3 = 1)
            P[4, i, j, 0] = V0 / math.sqrt(gphph)
    loc = np.arange(n1 * n2, dtype=np.int32)
    U = og.prim2cons(P.reshape(8, -1), loc).reshape((9,) + og.shape)
    og.set_state(P, U, 0.0, 1e-3)
    return og


def _closed_form(og):
    r = og.r_of_x1(og.x1in + (og.i_h + 0.5) * og.dx[0])
    alpha = 1.0 / math.sqrt(1.0 + 2.0 / r)
    w = RHO + GAM * UU
    return -2.0 * math.pi ** 2 * w * math.sqrt(1.0 + V0 * V0) * alpha * V0 * r * r


@pytest.mark.parametrize("n2", [16, 32, 64])
def test_ldot_equals_the_closed_form(n2):
    og = _grid(n2)
    ref = _closed_form(og)
    got = og.diagnostics()["ldot"]
    assert abs(got - ref) < 1e-13 * abs(ref), (got, ref)


def test_ldot_sign_follows_the_rotation():
    og = _grid(32)
    P, U, t, dt = og.get_state()
    P[4] *= -1.0
    loc = np.arange(P[0].size, dtype=np.int32)
    U = og.prim2cons(P.reshape(8, -1), loc).reshape(U.shape)
    og2 = _grid(32)
    og2.set_state(P, U, t, dt)
    assert og2.diagnostics()["ldot"] == pytest.approx(-og.diagnostics()["ldot"], rel=1e-14)
    # Mdot and Edot do not see the direction of rotation
    assert og2.diagnostics()["mdot"] == pytest.approx(og.diagnostics()["mdot"], rel=1e-14)
