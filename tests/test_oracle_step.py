"""Pins of the oracle step (Section 2.2, Eqs. 13-27; Section 2.3-2.4 fixups and floors).

- Flux-CT keeps the corner divergence of Eq. 24 at round-off (Kerr torus, 2D and 3D).
- Flat space, periodic box: the finite-volume update conserves every
  component of sum(U) to round-off (fluxes telescope, no source).
- Flat space: a small-amplitude relativistic sound wave moves at
  c_s^2 = gam p / (rho + u + p) and the scheme converges at second order.
- Failed inversions are replaced by the average of the four face
  neighbours, or the four diagonal neighbours (Eq. 33), exactly.
- Density / energy floors of Eq. 34 are applied exactly.
"""
import numpy as np
import pytest

import oracle

GAM = 4.0 / 3.0


def _flat_grid(n1, n2, n3, bc=oracle.BC_PERIODIC, **kw):
    p = oracle.default_params(metric=oracle.MINK_CART, n1=n1, n2=n2, n3=n3, x1min=0.0, x1max=1.0,
                              x2min=0.0, x2max=1.0, x3min=0.0, x3max=1.0, bc1=bc, bc2=bc, bc3=bc,
                              gam=GAM, **kw)
    return oracle.Grid(p)


def _centres(G):
    n1, n2, n3 = G.shape
    x = G.x1in + (np.arange(n1) + 0.5) * G.dx[0]
    y = G.x2in + (np.arange(n2) + 0.5) * G.dx[1]
    z = G.x3in + (np.arange(n3) + 0.5) * G.dx[2]
    return np.meshgrid(x, y, z, indexing="ij")


def _set_prims(G, P):
    n = P[0].size
    loc = np.zeros(n, dtype=np.int32)
    U = G.prim2cons(P.reshape(8, -1), loc)
    G.set_state(P, U, 0.0, 0.0)
    return U.reshape((9,) + G.shape)


@pytest.mark.parametrize("n3", [1, 6])
def test_flux_ct_keeps_divergence_at_roundoff(n3):
    p = oracle.default_params(n1=32, n2=32, n3=n3, gam=13.0 / 9.0)
    G = oracle.Grid(p)
    G.init_torus(pert_amp=0.04, seed=3)
    scale = None
    for _ in range(6):
        assert G.step() == 0
        P, U, t, dt = G.get_state()
        scale = np.abs(U[5:8]).max() / min(G.dx[0], G.dx[1])
        assert G.diagnostics()["divb_max"] <= 1e-13 * scale
    assert np.abs(U[7]).max() > 0 or n3 == 1


def test_flat_space_conservation():
    G = _flat_grid(12, 10, 8)
    X, Y, Z = _centres(G)
    tp = 2 * np.pi
    P = np.zeros((8,) + G.shape)
    P[0] = 1.0 + 0.3 * np.sin(tp * X) * np.cos(tp * Y)
    P[1] = 0.6 + 0.2 * np.cos(tp * (X + Z))
    P[2] = 0.3 * np.sin(tp * Y)
    P[3] = -0.2 * np.cos(tp * Z)
    P[4] = 0.25 * np.sin(tp * (X - Y))
    P[5] = 0.2 + 0.1 * np.sin(tp * Y)
    P[6] = 0.1 * np.cos(tp * Z)
    P[7] = 0.15 * np.sin(tp * X)
    U0 = _set_prims(G, P)
    G.set_dt(G.initial_dt())
    for _ in range(3):
        assert G.step() == 0
    U1 = G.get_state()[1]
    d = G.diagnostics()
    assert d["n_fail"] == 0 and d["n_floor"] == 0
    for c in range(9):
        s0, s1 = U0[c].sum(), U1[c].sum()
        assert abs(s1 - s0) <= 1e-13 * np.abs(U0[c]).sum(), c


def _sound_wave_error(n, amp=1e-6):
    G = _flat_grid(n, 1, 1)
    X = _centres(G)[0]
    rho0, u0 = 1.0, 1.0
    p0 = (GAM - 1) * u0
    w0 = rho0 + u0 + p0
    cs = np.sqrt(GAM * p0 / w0)
    # right-moving linear wave: drho = A rho, du = A (u + p), v = A cs
    prof = lambda x: np.sin(2 * np.pi * x)
    P = np.zeros((8,) + G.shape)
    P[0] = rho0 * (1 + amp * prof(X))
    P[1] = u0 + amp * (u0 + p0) * prof(X)
    v = amp * cs * prof(X)
    P[2] = v / np.sqrt(1 - v * v)
    _set_prims(G, P)
    t_end = 0.5 / cs
    nsteps = int(np.ceil(t_end / (0.3 * G.dx[0])))
    dt = t_end / nsteps
    for _ in range(nsteps):
        G.set_dt(dt)
        G.step()
    Pn, _, t, _ = G.get_state()
    assert t == pytest.approx(t_end, rel=1e-12)
    exact = rho0 * (1 + amp * prof(X - cs * t_end))
    return np.abs(Pn[0] - exact).mean() / amp


def test_sound_wave_second_order():
    e = [_sound_wave_error(n) for n in (32, 64, 128)]
    assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.3, e
    assert e[2] < 2e-3


def test_failed_zone_replaced_by_face_then_diagonal_average():
    G = _flat_grid(8, 8, 1)
    X, Y, Z = _centres(G)
    P = np.zeros((8,) + G.shape)
    P[0] = 1.0 + 0.3 * np.sin(2 * np.pi * X) + 0.1 * Y
    P[1] = 0.5 + 0.1 * np.cos(2 * np.pi * Y)
    P[2] = 0.1 * X
    P[3] = -0.05 * Y
    P[5] = 0.1
    U = _set_prims(G, P)
    Ubad = U.copy()
    Ubad[0, 3, 4, 0] = -1.0           # single failure -> face average
    Ubad[0, 5, 2, 0] = -1.0           # two adjacent failures -> diagonal averages
    Ubad[0, 6, 2, 0] = -1.0
    G.set_state(P, Ubad, 0.0, 0.0)
    nfl = G.invert_all()
    assert nfl == 3
    Pn = G.get_state()[0]
    face = lambda i, j: 0.25 * (P[:5, i + 1, j, 0] + P[:5, i - 1, j, 0] + P[:5, i, j + 1, 0] + P[:5, i, j - 1, 0])
    diag = lambda i, j: 0.25 * (P[:5, i + 1, j + 1, 0] + P[:5, i + 1, j - 1, 0] + P[:5, i - 1, j + 1, 0] +
                                P[:5, i - 1, j - 1, 0])
    assert np.allclose(Pn[:5, 3, 4, 0], face(3, 4), rtol=1e-13, atol=1e-14)
    assert np.allclose(Pn[:5, 5, 2, 0], diag(5, 2), rtol=1e-13, atol=1e-14)
    assert np.allclose(Pn[:5, 6, 2, 0], diag(6, 2), rtol=1e-13, atol=1e-14)
    # B untouched, U recomputed from the fixed primitives
    assert np.array_equal(Pn[5:8, 3, 4, 0], P[5:8, 3, 4, 0])
    Un = G.get_state()[1]
    assert Un[0, 3, 4, 0] > 0


def test_floors_exact():
    p = oracle.default_params(n1=16, n2=16, n3=1, gam=GAM)
    G = oracle.Grid(p)
    G.init_torus(pert_amp=0.0)
    P, U, t, dt = G.get_state()
    i, j = 5, 3
    r = G.r_of_x1(G.x1in + (i + 0.5) * G.dx[0])
    P[0, i, j, 0] = 1e-3 * 1e-5 * r ** -0.5
    P[1, i, j, 0] = 1e-3 * (1e-5 / 3) * r ** -2.5
    loc = np.repeat(np.arange(16 * 16, dtype=np.int32), 1)
    U = G.prim2cons(P.reshape(8, -1), loc).reshape(U.shape)
    G.set_state(P, U, t, dt)
    G.invert_all()
    Pn = G.get_state()[0]
    assert Pn[0, i, j, 0] == pytest.approx(1e-5 * r ** -0.5, rel=1e-14)
    assert Pn[1, i, j, 0] == pytest.approx((1e-5 / 3) * r ** -2.5, rel=1e-14)


def test_horizon_flux_of_split_monopole_closed_form():
    """phi_B = 1/2 sum |sqrt(-g) B^1| dX2 dX3 (Eq. 39) of a split monopole
    sqrt(-g) B^1 = +-B0 is 2 pi B0 exactly, and its corner divergence is 0."""
    p = oracle.default_params(n1=24, n2=24, n3=3, gam=GAM)
    G = oracle.Grid(p)
    G.init_torus(pert_amp=0.0, beta0=0.0)
    P, U, t, dt = G.get_state()
    tab = G.geom_table(0)
    gdet = tab[oracle.NG:oracle.NG + 24, oracle.NG:oracle.NG + 24, 32][:, :, None]
    sgn = np.where(np.arange(24) < 12, 1.0, -1.0)[None, :, None]
    B0 = 3e-3
    P[5] = B0 * sgn / gdet
    loc = np.repeat((np.arange(24)[:, None] * 24 + np.arange(24)[None, :]).astype(np.int32), 3, axis=1)
    U = G.prim2cons(P.reshape(8, -1), loc.reshape(-1)).reshape(U.shape)
    G.set_state(P, U, t, dt)
    d = G.diagnostics()
    assert d["phib"] == pytest.approx(2 * np.pi * B0, rel=1e-12)
    assert d["divb_max"] <= 1e-14 * B0 / G.dx[0]
    assert d["PhiB"] == pytest.approx(d["phib"] / np.sqrt(abs(d["mdot"])), rel=1e-12)
