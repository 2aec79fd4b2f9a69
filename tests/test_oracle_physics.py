"""Pins of the oracle pointwise physics (Sections 2.1-2.2).

Each pin is fixed by something other than the oracle's own formula:
normalisation identities of u^mu and b^mu, the closed-form stress tensor of a
fluid at rest in flat space, relativistic velocity addition for the wave
speeds of Eq. 19 and a brute-force minmod table for the MC limiter of Eq.
16.  The Riemann fluxes (Eqs. 18, 21) are pinned in test_oracle_limits.py.
"""
import numpy as np
import pytest

import oracle
from tests import inputs

GAM = 4.0 / 3.0


def _flat():
    return oracle.geom_from(np.diag([-1.0, 1.0, 1.0, 1.0]))


def _kerr_points(n=40, seed=3):
    p = oracle.default_params(n1=32, n2=32, n3=1, r_out=1000.0)
    G = oracle.Grid(p)
    tab = G.geom_table(0)
    loc = inputs.zone_locations(n, 32, 32, seed)
    geos = []
    for L in loc:
        i, j = divmod(int(L), 32)
        row = tab[i + oracle.NG, j + oracle.NG]
        geos.append(oracle.geom_from(row[:16].reshape(4, 4)))
    return geos


def test_four_velocity_and_field_identities():
    geos = _kerr_points()
    pp = inputs.prim_params(len(geos), seed=11)
    gsp = np.stack([np.array(g.gcov[:]).reshape(4, 4)[1:, 1:] for g in geos])
    P = inputs.place_prims(pp, gsp)
    for a, g in enumerate(geos):
        s, _ = oracle.state_of(P[:, a], g)
        gc = np.array(g.gcov[:]).reshape(4, 4)
        assert abs(s["ucon"] @ gc @ s["ucon"] + 1.0) < 1e-11 * s["gamma"] ** 2
        assert abs(s["ucon"] @ s["bcov"]) < 1e-11 * (1 + np.abs(s["ucon"]) @ np.abs(s["bcov"]))
        assert abs(s["gamma"] - pp["lorentz"][a]) < 1e-12 * pp["lorentz"][a]
        # B^i = b^i u^t - b^t u^i (Section 2.1)
        Brec = s["bcon"][1:] * s["ucon"][0] - s["bcon"][0] * s["ucon"][1:]
        assert np.allclose(Brec, P[5:8, a], rtol=1e-10, atol=1e-12 * np.abs(P[5:8, a]).max())


def test_flat_rest_frame_closed_forms():
    g = _flat()
    rho, u, B = 0.7, 0.3, np.array([0.2, -0.1, 0.4])
    q = np.array([rho, u, 0, 0, 0, *B])
    U = oracle.prim_to_U(q, g, GAM)
    p = (GAM - 1) * u
    bsq = B @ B
    # T^t_t = -(rho + u + b^2/2) at rest, momenta zero, entropy p / rho^(gam-1)
    assert np.allclose(U[:5], [rho, -(rho + u + 0.5 * bsq), 0, 0, 0], rtol=1e-15, atol=1e-15)
    assert np.allclose(U[5:8], B)
    assert abs(U[8] - p / rho ** (GAM - 1)) < 1e-15
    # flux along x at rest: momentum flux = p + b^2/2 - B_x^2, induction B_x terms vanish
    F = oracle.prim_to_F(q, g, GAM, 1)
    assert abs(F[2] - (p + 0.5 * bsq - B[0] ** 2)) < 1e-15
    assert abs(F[3] + B[0] * B[1]) < 1e-15 and abs(F[4] + B[0] * B[2]) < 1e-15
    assert F[0] == 0.0 and F[5] == 0.0


def _cs(rho, u):
    p = (GAM - 1) * u
    return np.sqrt(GAM * p / (rho + u + p))


@pytest.mark.parametrize("v", [0.0, 0.3, -0.6, 0.95])
def test_wave_speeds_velocity_addition(v):
    g = _flat()
    rho, u = 1.0, 0.5
    lor = 1 / np.sqrt(1 - v * v)
    q = np.array([rho, u, lor * v, 0, 0, 0, 0, 0])
    c1, c2 = oracle.wave_speeds(q, g, GAM, 1)
    cs = _cs(rho, u)
    assert abs(c1 - (v + cs) / (1 + v * cs)) < 1e-14
    assert abs(c2 - (v - cs) / (1 - v * cs)) < 1e-14
    # transverse direction of a flow along x: +- cs / Gamma-contracted (quadratic symmetric)
    c1y, c2y = oracle.wave_speeds(q, g, GAM, 2)
    assert abs(c1y + c2y) < 1e-14


def test_wave_speeds_magnetised_rest():
    g = _flat()
    rho, u, B = 1.0, 0.5, np.array([0.3, 0.4, 0.0])
    q = np.array([rho, u, 0, 0, 0, *B])
    p = (GAM - 1) * u
    bsq = B @ B
    va2 = bsq / (bsq + rho + u + p)
    cs2 = _cs(rho, u) ** 2
    cms = np.sqrt(va2 + cs2 * (1 - va2))
    for d in (1, 2, 3):
        c1, c2 = oracle.wave_speeds(q, g, GAM, d)
        assert abs(c1 - cms) < 1e-14 and abs(c2 + cms) < 1e-14


def _minmod3(a, b, c):
    if a > 0 and b > 0 and c > 0:
        return min(a, b, c)
    if a < 0 and b < 0 and c < 0:
        return max(a, b, c)
    return 0.0


def test_mc_limiter_brute_force():
    vals = np.array([-3.0, -1.0, -0.25, 0.0, 0.5, 1.0, 2.0, 7.0])
    for qm in vals:
        for q0 in vals:
            for qp in vals:
                ref = _minmod3(2 * (q0 - qm), 2 * (qp - q0), 0.5 * (qp - qm))
                assert oracle.mc_slope(qm, q0, qp) == pytest.approx(ref, abs=1e-15), (qm, q0, qp)


def test_face_reconstruction_bounded():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        q = rng.normal(size=4)
        ql = q[1] + 0.5 * oracle.mc_slope(q[0], q[1], q[2])
        qr = q[2] - 0.5 * oracle.mc_slope(q[1], q[2], q[3])
        lo, hi = min(q[1], q[2]), max(q[1], q[2])
        assert lo - 1e-15 <= ql <= hi + 1e-15 and lo - 1e-15 <= qr <= hi + 1e-15
