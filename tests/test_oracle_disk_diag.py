"""The oracle's barycentric radius (Eq. 43) pinned by closed forms: for a
uniform density the ratio is the same ratio of radial integrals of the
Kerr-Schild volume element sqrt(-g) = (r^2 + a^2 cos^2 theta) sin theta,

  int int r sqrt(-g) dtheta dphi = 2 pi r (2 r^2 + 2 a^2 / 3),

over the radial range the included zones cover (from the lower face of the
horizon zone to the upper face of the last zone whose centre is at most
r_bar_max); the midpoint sums of the code coordinates converge to it at
second order."""
import numpy as np
import pytest

import oracle as O


def _uniform(n1, n2, a, rho=1.0):
    og = O.Grid(O.default_params(n1=n1, n2=n2, n3=1, a=a, r_out=40.0))
    P = np.zeros((8,) + og.shape)
    P[0], P[1] = rho, 1e-2  # at rest in the normal frame (ut^i = 0), no field
    loc = np.repeat(np.arange(n1 * n2, dtype=np.int32), 1)
    U = og.prim2cons(P.reshape(8, -1), loc).reshape((9,) + og.shape)
    og.set_state(P, U, 0.0, 1e-3)
    return og


def _closed_form(og, r_bar_max, a):
    n1 = og.shape[0]
    rc = [og.r_of_x1(og.x1in + (i + 0.5) * og.dx[0]) for i in range(n1)]
    i1 = max(i for i in range(n1) if rc[i] <= r_bar_max)
    ra = og.r_of_x1(og.x1in + og.i_h * og.dx[0])
    rb = og.r_of_x1(og.x1in + (i1 + 1) * og.dx[0])
    N = lambda r: r ** 4 / 2.0 + a * a * r * r / 3.0
    D = lambda r: 2.0 * r ** 3 / 3.0 + 2.0 * a * a * r / 3.0
    return (N(rb) - N(ra)) / (D(rb) - D(ra)), 2.0 * np.pi * (D(rb) - D(ra))


@pytest.mark.parametrize("a", [0.0, 0.9375])
def test_barycentric_radius_converges_to_the_closed_form(a):
    errs, merrs = [], []
    for n1, n2 in ((32, 16), (64, 32), (128, 64)):
        og = _uniform(n1, n2, a)
        rbar, mass, num = og.barycentric(30.0)
        exact, mass_exact = _closed_form(og, 30.0, a)
        errs.append(abs(rbar / exact - 1.0))
        merrs.append(abs(mass / mass_exact - 1.0))
        assert rbar == pytest.approx(num / mass, rel=1e-15)
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    assert merrs[0] / merrs[1] > 3.5 and merrs[1] / merrs[2] > 3.5, merrs
    assert errs[2] < 3e-4 and merrs[2] < 1.5e-4, (errs, merrs)


def test_barycentric_radius_is_density_weighted():
    """Scaling rho scales both sums and leaves <r> unchanged; mass moved
    outward moves <r> outward; zones beyond r_bar_max do not count."""
    og = _uniform(48, 16, 0.9375)
    r1, m1, _ = og.barycentric(25.0)
    og2 = _uniform(48, 16, 0.9375, rho=3.0)
    r2, m2, _ = og2.barycentric(25.0)
    assert r2 == pytest.approx(r1, rel=1e-14) and m2 == pytest.approx(3.0 * m1, rel=1e-14)
    P, U, t, dt = og.get_state()
    rc = np.array([og.r_of_x1(og.x1in + (i + 0.5) * og.dx[0]) for i in range(48)])
    P[0][rc > 15.0] *= 2.0
    og.set_state(P, U, t, dt)
    assert og.barycentric(25.0)[0] > r1
    P[0][rc > 25.0] *= 100.0
    og.set_state(P, U, t, dt)
    r3 = og.barycentric(25.0)[0]
    P[0][rc > 25.0] /= 100.0
    og.set_state(P, U, t, dt)
    assert og.barycentric(25.0)[0] == r3
