"""Pins of the oracle's polar cylindrification (Section 4.1 cylindrifies the
cells next to the poles after Tchekhovskoy et al. 2011 and prints no
formula; the reading, a widening of the rows next to each pole by
lambda(r) = (1 + (r_c/r)^4)^(1/4) inside a band of X2 width y_b, is written
out in oracle/geometry.c).

Fixed by things other than the oracle's own formulas:
  * the partial derivatives of theta(X1, X2) against central differences of
    theta itself, in both bands, beyond the poles (ghost rows) and across
    the band edges;
  * the poles stay on the axis, outside the bands the angle is Eq. 36 to
    the bit, the map is monotone in X2 at every radius, it is symmetric
    about the equator and odd about each pole (the mirror the polar
    boundary uses), and at a pole d theta/dX2 is lambda(r) times the MKS
    value -- lambda written here from its definition;
  * the code metric against the tensor transformation law g = J^T g_KS J
    with J from central differences of r(X1) and theta(X1, X2), sqrt(-g)
    against numpy's determinant, g^{mn} against numpy's inverse, and the
    connection against central differences of the metric;
  * Michel's steady accretion flow (an exact solution that does not know
    the grid) is held with second-order convergence on a cylindrified grid,
    where it has u^2 != 0 inside the bands;
  * flux-CT keeps the corner divergence at round-off, and the 3D torus CFL
    step grows (the point of the transformation).
"""
import math

import numpy as np
import pytest

import oracle as O
from tests.michel import Michel, michel_prims

A = 0.9375
H = 0.3


def _grid(n1=32, n2=32, n3=1, cyl_r=2.2, cyl_dx2=0.25, **kw):
    return O.Grid(O.default_params(n1=n1, n2=n2, n3=n3, cyl_r=cyl_r, cyl_dx2=cyl_dx2, **kw))


def _lam(r, rc):
    return (1.0 + (rc / r) ** 4) ** 0.25


def _points(G):
    X1s = [G.x1in - 2.5 * G.dx[0], G.x1in, G.x1in + 0.7, G.x1in + 2.0, G.x1in + 3.2]
    X2s = [-1.05, -1.01, -0.99, -0.93, -0.88, -0.8, -0.76, -0.749, -0.6, 0.2,
           0.77, 0.8, 0.9, 0.97, 1.0 - 1e-3, 1.02]
    return [(a, b) for a in X1s for b in X2s]


def test_partials_against_central_differences():
    G = _grid()
    h = 1e-6
    for X1, X2 in _points(G):
        th, d1, d2 = G.theta_at(X1, X2)
        f1 = (G.theta_at(X1 + h, X2)[0] - G.theta_at(X1 - h, X2)[0]) / (2 * h)
        f2 = (G.theta_at(X1, X2 + h)[0] - G.theta_at(X1, X2 - h)[0]) / (2 * h)
        assert abs(d1 - f1) < 2e-8 * (1.0 + abs(d2)), (X1, X2, d1, f1)
        assert abs(d2 - f2) < 2e-8 * (1.0 + abs(d2)), (X1, X2, d2, f2)


def test_axis_band_symmetry_and_monotone():
    G = _grid()
    M = _grid(cyl_r=0.0)
    yb = 0.25
    for X1 in (G.x1in - 2 * G.dx[0], G.x1in, G.x1in + 1.0, G.x1in + 3.0):
        r = G.r_of_x1(X1)
        assert G.theta_at(X1, -1.0)[0] == 0.0
        assert G.theta_at(X1, 1.0)[0] == pytest.approx(math.pi, abs=1e-15)
        # at a pole d theta/dX2 = lambda(r) * d theta_MKS/dX2 = lambda (2 - h) pi / 2
        d2 = G.theta_at(X1, -1.0)[2]
        assert d2 == pytest.approx(_lam(r, 2.2) * (2.0 - H) * math.pi / 2, rel=1e-13)
        X2 = np.linspace(-1.0 - 2.5 * G.dx[1], 1.0 + 2.5 * G.dx[1], 4001)
        th = np.array([G.theta_at(X1, x)[0] for x in X2])
        assert np.all(np.diff(th) > 0.0)
        assert np.all(np.array([G.theta_at(X1, x)[2] for x in X2]) > 0.0)
        for x in X2:
            t, d1, d2 = G.theta_at(X1, x)
            if abs(x) <= 1.0 - yb or abs(x) >= 1.0 + yb:
                assert t == M.theta_at(X1, x)[0] and d1 == 0.0      # MKS to the bit
            tm, e1, e2 = G.theta_at(X1, -x)
            assert t + tm == pytest.approx(math.pi, abs=1e-14)       # equatorial symmetry
            assert d1 == pytest.approx(-e1, abs=1e-14) and d2 == pytest.approx(e2, rel=1e-14)
        for t0 in (0.003, 0.02, 0.1, 0.2):                           # odd about each pole
            a = G.theta_at(X1, -1.0 + t0)
            b = G.theta_at(X1, -1.0 - t0)
            assert b[0] == pytest.approx(-a[0], abs=1e-15)
            assert b[1] == pytest.approx(-a[1], abs=1e-15) and b[2] == pytest.approx(a[2], rel=1e-13)
    # far out the grid is MKS again (lambda -> 1): the widening fades with r
    X1 = G.x1_of_r(40.0)
    assert abs(G.theta_at(X1, -0.95)[0] - M.theta_at(X1, -0.95)[0]) < 2e-4


def _J_fd(G, X1, X2, h=1e-6):
    """dx^a/dX^m from central differences of r(X1) and theta(X1, X2)."""
    J = np.zeros((4, 4))
    J[0, 0] = J[3, 3] = 1.0
    J[1, 1] = (G.r_of_x1(X1 + h) - G.r_of_x1(X1 - h)) / (2 * h)
    J[2, 1] = (G.theta_at(X1 + h, X2)[0] - G.theta_at(X1 - h, X2)[0]) / (2 * h)
    J[2, 2] = (G.theta_at(X1, X2 + h)[0] - G.theta_at(X1, X2 - h)[0]) / (2 * h)
    return J


def test_metric_is_the_transformed_kerr_schild_metric():
    G = _grid(n1=64, r_out=1000.0)
    for X1, X2 in _points(G):
        if abs(X2) >= 1.0:
            continue
        r, th = G.r_of_x1(X1), G.theta_at(X1, X2)[0]
        gks = O.ks_gcov(r, th, A)
        J = _J_fd(G, X1, X2)
        want = J.T @ gks @ J
        geo = G.geom_at(X1, X2)
        gcov = np.array(geo.gcov[:]).reshape(4, 4)
        gcon = np.array(geo.gcon[:]).reshape(4, 4)
        s = np.abs(want).max()
        assert np.abs(gcov - want).max() < 1e-8 * s, (X1, X2)
        assert geo.gdet == pytest.approx(math.sqrt(-np.linalg.det(gcov)), rel=1e-11)
        inv = np.linalg.inv(gcov)
        assert np.abs(gcon - inv).max() < 1e-10 * np.abs(inv).max(), (X1, X2)
        assert geo.alpha == pytest.approx(1.0 / math.sqrt(-inv[0, 0]), rel=1e-12)


def test_connection_against_differences_of_the_metric():
    G = _grid(n1=64, r_out=1000.0)
    h = 1e-5

    def gcov(X1, X2):
        return np.array(G.geom_at(X1, X2).gcov[:]).reshape(4, 4)

    for X1, X2 in [(G.x1in + 0.05, -0.97), (G.x1in + 0.4, -0.9), (G.x1in + 0.9, -0.8),
                   (G.x1in + 0.2, 0.85), (G.x1in + 1.5, 0.95)]:
        dg = np.zeros((4, 4, 4))
        dg[1] = (gcov(X1 + h, X2) - gcov(X1 - h, X2)) / (2 * h)
        dg[2] = (gcov(X1, X2 + h) - gcov(X1, X2 - h)) / (2 * h)
        gi = np.linalg.inv(gcov(X1, X2))
        want = 0.5 * (np.einsum("ls,msn->lmn", gi, dg) + np.einsum("ls,nsm->lmn", gi, dg)
                      - np.einsum("ls,smn->lmn", gi, dg))
        got = G.conn_at(X1, X2)
        assert np.abs(got - want).max() < 1e-6 * np.abs(want).max(), (X1, X2)
        # d theta/dX1 != 0 puts X1-X2 cross terms in the metric, hence Gamma^l_{12}
        assert np.abs(got[:, 1, 2]).max() > 1e-3 * np.abs(got).max()


@pytest.mark.parametrize("kw", [dict(cyl_r=5.0), dict(cyl_dx2=0.0), dict(cyl_dx2=1.2),
                                dict(cyl_r=float("inf")),
                                dict(metric=O.MINK_CART, x1min=0.0, x1max=1.0, x2min=0.0, x2max=1.0)])
def test_refused_parameters(kw):
    with pytest.raises(ValueError):
        _grid(**kw)


def _michel_drift(n1, n2, t_end=4.0):
    mic = Michel(r_c=8.0, n=3.0)
    gam = 4.0 / 3.0
    # r_c = 3.5: lambda = 1.83 at the horizon, 1.3 at r = 3
    og = O.Grid(O.default_params(n1=n1, n2=n2, n3=1, a=0.0, r_out=20.0, gam=gam, cyl_r=3.5, cyl_dx2=0.5))
    P0 = michel_prims(og, mic, gam)
    loc = np.repeat((np.arange(n1)[:, None] * n2 + np.arange(n2)[None, :]).reshape(-1), 1).astype(np.int32)
    U = og.prim2cons(P0.reshape(8, -1), loc).reshape((9,) + og.shape)
    og.set_state(P0, U, 0.0, 0.0)
    og.set_dt(og.initial_dt())
    while True:
        _, _, t, dt = og.get_state()
        if t >= t_end - 1e-12:
            break
        if t + dt > t_end:
            og.set_dt(t_end - t)
        assert og.step() == 0
    P = og.get_state()[0]
    r = np.array([og.r_of_x1(og.x1in + (i + 0.5) * og.dx[0]) for i in range(n1)])
    X2 = og.x2in + (np.arange(n2) + 0.5) * og.dx[1]
    rows = np.abs(X2) > 0.5          # the two bands
    band = (r > 3.0) & (r < 12.0)
    return np.abs(P[0][np.ix_(band, rows)][..., 0] / P0[0][np.ix_(band, rows)][..., 0] - 1.0).mean(), P0


def test_michel_flow_held_at_second_order_on_a_cylindrified_grid():
    e = []
    for n1, n2 in ((32, 8), (64, 16), (128, 32)):
        err, P0 = _michel_drift(n1, n2)
        e.append(err)
        assert np.abs(P0[3]).max() > 0.0       # the radial flow has u^2 != 0 in the bands
    print("cylindrified Michel drift", e)
    # the coarsest grid has two rows per band (ratio 2.9); 256 x 64 continues
    # the sequence at 3.8, too slow to run here
    assert e[0] / e[1] > 2.5 and e[1] / e[2] > 3.5, e
    assert e[2] < 1e-3


def test_torus_divergence_and_dt():
    G = _grid(n1=32, n2=32, n3=4)
    G.init_torus(pert_amp=0.04, seed=3)
    for _ in range(4):
        assert G.step() == 0
        U = G.get_state()[1]
        scale = np.abs(U[5:8]).max() / min(G.dx[0], G.dx[1])
        assert G.diagnostics()["divb_max"] <= 1e-13 * scale
    # 3D: the CFL step is set near the pole at the horizon, where the rows
    # are now wider in phi
    dts = []
    for rc in (0.0, 2.2):
        g = _grid(n1=32, n2=32, n3=32, cyl_r=rc)
        g.init_torus(pert_amp=0.0)
        dts.append(g.initial_dt())
    print("3D torus dt: MKS", dts[0], "cylindrified", dts[1])
    assert dts[1] > 1.15 * dts[0]
