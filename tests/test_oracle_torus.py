"""Pins of the oracle initial state (Section 5, first paragraphs; Eq. 45).

- The paper's own printed numbers: Table 1 columns (11)-(12), initial disk
  mass M and magnetic energy E_B for runs R1, R3, R4, R7, R8, R9 (stored in
  tests/golden/table1_initial_disk.json with the citation).
- The pressure maximum of a Fishbone-Moncrief torus is a circular geodesic,
  so the fluid angular velocity there is Kepler's Omega = 1/(r^1.5 + a)
  (Bardeen, Press & Teukolsky 1972).
- Hydrostatic equilibrium d_i ln h = -1/2 u_mu u_nu d_i g^{mu nu}, with the
  closed-form Boyer-Lindquist inverse metric.
- The discrete curl of A_phi has zero corner divergence (Eq. 24); beta_0 is
  max p_g / max p_B; the splitmix64 generator matches its published output.
"""
import json
import os

import numpy as np
import pytest

import oracle

A = 0.9375
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_initial_disk.json")


@pytest.mark.parametrize("run", ["R1", "R3", "R4", "R7", "R8", "R9"])
def test_table1_initial_mass_and_magnetic_energy(run):
    g = json.load(open(GOLDEN))["runs"][run]
    p = oracle.default_params(n1=g["n_r"], n2=g["n_theta"], n3=1, gam=g["gamma"], r_out=5000.0)
    G = oracle.Grid(p)
    G.init_torus(r_in=6.0, r_max=g["r_max"], beta0=g["beta0"], pert_amp=0.0)
    d = G.diagnostics()
    # printed with 2-3 significant figures; the grid here has no polar
    # cylindrification, which does not touch the disk
    assert d["disk_mass"] == pytest.approx(g["M"], rel=0.02)
    assert d["disk_eb"] == pytest.approx(g["E_B"], rel=0.02)


@pytest.mark.parametrize("r_max", [12.0, 13.0, 20.0])
def test_pressure_maximum_is_keplerian(r_max):
    ell = oracle.fm_ell(A, r_max)
    u = oracle.fm_ucon_bl(A, ell, r_max, np.pi / 2)
    assert u[3] / u[0] == pytest.approx(1.0 / (r_max ** 1.5 + A), rel=1e-12)


def _bl_gcon(r, th):
    s2, c2 = np.sin(th) ** 2, np.cos(th) ** 2
    sig = r * r + A * A * c2
    dl = r * r - 2 * r + A * A
    AA = (r * r + A * A) ** 2 - dl * A * A * s2
    g = np.zeros((4, 4))
    g[0, 0] = -AA / (sig * dl)
    g[0, 3] = g[3, 0] = -2 * A * r / (sig * dl)
    g[3, 3] = (dl - A * A * s2) / (sig * dl * s2)
    g[1, 1] = dl / sig
    g[2, 2] = 1 / sig
    return g


@pytest.mark.parametrize("r,th", [(8.0, 1.5), (12.0, 1.3), (20.0, 1.6), (30.0, 1.45), (10.0, 1.9)])
def test_hydrostatic_equilibrium(r, th):
    ell = oracle.fm_ell(A, 12.0)
    u = oracle.fm_ucon_bl(A, ell, r, th)
    gi = _bl_gcon(r, th)
    ucov = np.linalg.solve(gi, u)
    assert ucov @ u == pytest.approx(-1.0, abs=1e-12)
    assert u[0] * ucov[3] == pytest.approx(ell, rel=1e-12)
    h = 1e-5
    dlnh_r = (oracle.fm_lnh(A, ell, r + h, th) - oracle.fm_lnh(A, ell, r - h, th)) / (2 * h)
    dlnh_t = (oracle.fm_lnh(A, ell, r, th + h) - oracle.fm_lnh(A, ell, r, th - h)) / (2 * h)
    dg_r = (_bl_gcon(r + h, th) - _bl_gcon(r - h, th)) / (2 * h)
    dg_t = (_bl_gcon(r, th + h) - _bl_gcon(r, th - h)) / (2 * h)
    assert dlnh_r == pytest.approx(-0.5 * ucov @ dg_r @ ucov, rel=1e-6, abs=1e-10)
    assert dlnh_t == pytest.approx(-0.5 * ucov @ dg_t @ ucov, rel=1e-6, abs=1e-10)


def test_initial_field_divergence_free_and_beta0():
    p = oracle.default_params(n1=48, n2=48, n3=2, gam=4.0 / 3.0)
    G = oracle.Grid(p)
    G.init_torus(r_in=6.0, r_max=12.0, beta0=100.0, pert_amp=0.0)
    P, U, t, dt = G.get_state()
    d = G.diagnostics()
    scale = np.abs(U[5:8]).max() / G.dx[:2].min()
    assert d["divb_max"] <= 1e-13 * scale
    assert np.abs(P[7]).max() == 0.0
    # beta_0 = max p_g / max b^2/2 (b^2 = 2 (p_g/beta) at the field maximum)
    tab = G.geom_table(0)
    pmax = ((4.0 / 3.0 - 1) * P[1]).max()
    bsq = []
    for i in range(48):
        for j in range(48):
            g = oracle.geom_from(tab[i + oracle.NG, j + oracle.NG, :16].reshape(4, 4))
            s, _ = oracle.state_of(P[:, i, j, 0], g)
            bsq.append(s["bsq"])
    assert pmax / (0.5 * max(bsq)) == pytest.approx(100.0, rel=1e-10)
    assert dt > 0 and np.isfinite(dt)


def test_splitmix64_published_output():
    # splitmix64 seeded with 0 first returns 0xE220A8397B1DCDAF
    xi = oracle.uniform(0, 0)
    assert xi == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53


def test_perturbation_amplitude_and_determinism():
    p = oracle.default_params(n1=32, n2=32, n3=4, gam=13.0 / 9.0)
    G0 = oracle.Grid(p)
    G0.init_torus(pert_amp=0.0)
    G1 = oracle.Grid(p)
    G1.init_torus(pert_amp=0.04, seed=1)
    G2 = oracle.Grid(p)
    G2.init_torus(pert_amp=0.04, seed=1)
    P0, P1, P2 = G0.get_state()[0], G1.get_state()[0], G2.get_state()[0]
    assert np.array_equal(P1, P2)
    torus = P0[0] > 0.01
    ratio = P1[1][torus] / P0[1][torus]
    assert ratio.min() >= 0.96 and ratio.max() <= 1.04 and ratio.std() > 0.01
    assert np.array_equal(P0[0], P1[0])


def _torus_drift(n, t_end=10.0):
    """Mean relative change of rho in the torus body after t_end of the
    unmagnetised, unperturbed Fishbone-Moncrief torus (an equilibrium)."""
    p = oracle.default_params(n1=n, n2=n, n3=1, a=0.9375, r_out=40.0, gam=4.0 / 3.0)
    og = oracle.Grid(p)
    og.init_torus(r_in=6.0, r_max=12.0, beta0=0.0, pert_amp=0.0, seed=1)
    P0 = og.get_state()[0].copy()
    while True:
        _, _, t, dt = og.get_state()
        if t >= t_end - 1e-12:
            break
        if t + dt > t_end:
            og.set_dt(t_end - t)
        assert og.step() == 0
    P = og.get_state()[0]
    r = np.array([og.r_of_x1(og.x1in + (i + 0.5) * og.dx[0]) for i in range(n)])
    th = np.array([og.th_of_x2(og.x2in + (j + 0.5) * og.dx[1]) for j in range(n)])
    R, TH = np.meshgrid(r, th, indexing="ij")
    body = (R > 9.0) & (R < 16.0) & (np.abs(TH - np.pi / 2) < 0.25)
    return np.abs(P[0, :, :, 0][body] / P0[0, :, :, 0][body] - 1.0).mean()


def test_unmagnetised_torus_is_stationary_to_second_order():
    # the whole step (fluxes, Kerr connection sources, RK2, inversion) keeps
    # the equilibrium up to truncation error, which falls at second order
    e32, e64 = _torus_drift(32), _torus_drift(64)
    assert e32 / e64 > 3.0, (e32, e64)
    assert e64 < 1e-3
