"""Pins of the oracle geometry (Section 4.1, Eqs. 35-36) against closed forms.

Pinned by textbook identities that share no formula with the oracle code:
the Kerr-Schild inverse metric and determinant in closed form, the Kepler
law Omega = 1/(r^1.5 + a) of circular equatorial geodesics (Bardeen, Press
& Teukolsky 1972) through the connection, and flat space.
"""
import numpy as np
import pytest

import oracle

A = 0.9375


def _ks_closed_inverse(r, th, a):
    sig = r * r + a * a * np.cos(th) ** 2
    delta = r * r - 2 * r + a * a
    gi = np.zeros((4, 4))
    gi[0, 0] = -(1 + 2 * r / sig)
    gi[0, 1] = gi[1, 0] = 2 * r / sig
    gi[1, 1] = delta / sig
    gi[1, 3] = gi[3, 1] = a / sig
    gi[2, 2] = 1 / sig
    gi[3, 3] = 1 / (sig * np.sin(th) ** 2)
    return gi, sig * np.sin(th)


@pytest.mark.parametrize("r,th", [(1.5, 0.3), (2.0, 1.2), (6.0, np.pi / 2), (40.0, 2.9), (900.0, 0.01)])
def test_ks_inverse_and_determinant_closed_form(r, th):
    g = oracle.ks_gcov(r, th, A)
    gi, sqrtg = _ks_closed_inverse(r, th, A)
    geo = oracle.geom_from(g)
    gcon = np.array(geo.gcon[:]).reshape(4, 4)
    scale = np.abs(gi).max()
    assert np.abs(gcon - gi).max() <= 1e-12 * scale
    assert abs(geo.gdet - sqrtg) <= 1e-13 * sqrtg
    assert np.abs(g @ gcon - np.eye(4)).max() < 1e-12


def _grid(**kw):
    p = oracle.default_params(n1=16, n2=16, n3=4, **kw)
    return oracle.Grid(p)


def test_mks_map_and_jacobian():
    G = _grid(r_out=1000.0)
    assert abs(G.th_of_x2(0.0) - np.pi / 2) < 1e-15
    assert abs(G.th_of_x2(-1.0)) < 1e-15 and abs(G.th_of_x2(1.0) - np.pi) < 1e-14
    # r(X1) continuous with continuous derivative across the break at 400 M
    xb = np.log(400.0)
    for x in (xb - 1e-7, xb, xb + 1e-7):
        assert abs(G.r_of_x1(x) - np.exp(x)) < 1e-4
    # sqrt(-g) of MKS = Sigma sin(theta) r'(X1) theta'(X2), numerical Jacobian
    for X1, X2 in [(0.5, -0.4), (2.0, 0.1), (6.5, 0.7)]:
        geo = G.geom_at(X1, X2)
        r, th = G.r_of_x1(X1), G.th_of_x2(X2)
        h = 1e-6
        dr = (G.r_of_x1(X1 + h) - G.r_of_x1(X1 - h)) / (2 * h)
        dth = (G.th_of_x2(X2 + h) - G.th_of_x2(X2 - h)) / (2 * h)
        sig = r * r + A * A * np.cos(th) ** 2
        assert abs(geo.gdet - sig * np.sin(th) * dr * dth) < 1e-8 * geo.gdet
        # equator-refining: dtheta/dX2 = h pi / 2 at the equator
    dth0 = (G.th_of_x2(1e-6) - G.th_of_x2(-1e-6)) / 2e-6
    assert abs(dth0 - 0.3 * np.pi / 2) < 1e-8


def test_connection_symmetric_and_kepler_geodesic():
    G = _grid(r_out=1000.0)
    for r in (3.0, 6.0, 12.0, 50.0, 600.0):
        X1 = G.x1_of_r(r)
        conn = G.conn_at(X1, 0.0)
        assert np.abs(conn - conn.transpose(0, 2, 1)).max() <= 1e-13 * np.abs(conn).max()
        om = 1.0 / (r ** 1.5 + A)
        u = np.array([1.0, 0.0, 0.0, om])
        acc = np.einsum("lmn,m,n->l", conn, u, u)
        terms = np.einsum("lmn,m,n->lmn", np.abs(conn), np.abs(u), np.abs(u)).sum(axis=(1, 2))
        # radial and polar geodesic acceleration of a Kepler orbit vanish
        assert abs(acc[1]) <= 1e-12 * terms[1]
        assert abs(acc[2]) <= 1e-12 * terms[1]


def test_connection_matches_finite_difference_of_closed_form_metric():
    """Gamma from central differences of the closed-form KS metric mapped to MKS."""
    G = _grid(r_out=40.0)
    X1, X2 = 1.3, 0.37
    h = 1e-4

    def gmks(x1, x2):
        r, th = np.exp(x1), np.pi / 2 * (1 + x2) + 0.35 * np.sin(np.pi * (1 + x2))
        dr, dth = np.exp(x1), np.pi / 2 + 0.35 * np.pi * np.cos(np.pi * (1 + x2))
        sig = r * r + A * A * np.cos(th) ** 2
        z = 2 * r / sig
        s2 = np.sin(th) ** 2
        g = np.zeros((4, 4))
        g[0, 0] = -(1 - z)
        g[0, 1] = g[1, 0] = z
        g[0, 3] = g[3, 0] = -A * z * s2
        g[1, 1] = 1 + z
        g[1, 3] = g[3, 1] = -A * (1 + z) * s2
        g[2, 2] = sig
        g[3, 3] = s2 * (sig + A * A * (1 + z) * s2)
        J = np.array([1.0, dr, dth, 1.0])
        return g * np.outer(J, J)

    def d(f, i):
        e = np.zeros(2)
        e[i] = h
        c = [(-2, 1), (-1, -8), (1, 8), (2, -1)]
        return sum(w * f(X1 + s * e[0], X2 + s * e[1]) for s, w in c) / (12 * h)

    dg = np.zeros((4, 4, 4))
    dg[1] = d(gmks, 0)
    dg[2] = d(gmks, 1)
    gi = np.linalg.inv(gmks(X1, X2))
    ref = 0.5 * (np.einsum("ls,msn->lmn", gi, dg) + np.einsum("ls,nsm->lmn", gi, dg)
                 - np.einsum("ls,smn->lmn", gi, dg))
    conn = G.conn_at(X1, X2)
    assert np.abs(conn - ref).max() <= 1e-9 * np.abs(ref).max()


def test_flat_space_geometry():
    p = oracle.default_params(metric=oracle.MINK_CART, n1=8, n2=8, n3=8)
    G = oracle.Grid(p)
    geo = G.geom_at(0.3, 0.4)
    assert np.allclose(np.array(geo.gcov[:]).reshape(4, 4), np.diag([-1.0, 1, 1, 1]))
    assert geo.gdet == 1.0 and geo.alpha == 1.0
    assert np.abs(G.conn_at(0.3, 0.4)).max() == 0.0


def test_horizon_zone_index():
    G = _grid(r_out=40.0)
    rh = 1 + np.sqrt(1 - A * A)
    rc = [G.r_of_x1(G.x1in + (i + 0.5) * G.dx[0]) for i in range(16)]
    i_h = next(i for i, r in enumerate(rc) if r >= rh)
    assert G.i_h == i_h
