"""Pins of the oracle's piecewise parabolic reconstruction (the parabolic
method Section 2.2 names as the more accurate successor of its PLM; written
from Colella & Woodward 1984 for uniform zones, without contact steepening or
shock flattening).

Fixed by things other than the oracle's own formula:
  * the interface value of MC-limited slopes is the fourth-order
    interpolation of zone averages, exact for a cubic's cell averages where
    the limiter leaves the central slope and the monotonicity constraint is
    inactive (smooth, monotone data);
  * constant and linear data are reproduced, and a step stays a step;
  * brute force: every face state lies between the two zones beside it, and
    every zone's limited parabola (a_L, a, a_R) is monotone inside the zone
    -- |a - (a_L + a_R)/2| <= |a_R - a_L| / 6 and a between a_L and a_R --
    the property the constraint exists to give;
  * on a smooth relativistic sound wave in flat space the step with PPM
    converges at second order (the RK2 time integration limits it); the
    monotonicity constraint flattens the wave's smooth extrema, so there its
    error stays near PLM's;
  * on the shock tube (exact special-relativistic Riemann solution, the
    states of test_oracle_shocktube) PPM's L1 error is well below PLM's at
    every resolution: the discontinuities are what the parabolas sharpen.
"""
import numpy as np
import pytest

import oracle
from tests.test_oracle_step import GAM, _centres, _flat_grid, _set_prims


def _cubic_averages(h, coef, n=6):
    """Cell averages of f(x) = sum c_k x^k over zones of width h whose
    centres sit at (m - 2.5) h, m = 0..5 (the face between zones 2 and 3 at
    x = 0); f's antiderivative evaluated at the zone edges."""
    F = lambda x: sum(c * x ** (k + 1) / (k + 1) for k, c in enumerate(coef))
    edges = (np.arange(n + 1) - 3.0) * h
    return np.array([(F(edges[m + 1]) - F(edges[m])) / h for m in range(n)])


@pytest.mark.parametrize("h", [0.05, 0.01])
def test_cubic_cell_averages_give_the_exact_face_value(h):
    coef = (1.0, 3.0, 0.5, 1.0)   # 1 + 3x + x^2/2 + x^3: monotone near 0
    q = _cubic_averages(h, coef)
    ql, qr = oracle.ppm_face(q)
    assert ql == pytest.approx(1.0, abs=1e-14) and qr == pytest.approx(1.0, abs=1e-14)
    # PLM's face values are only second order: wrong by O(h^2)
    plm_l = q[2] + 0.5 * oracle.mc_slope(q[1], q[2], q[3])
    assert abs(plm_l - 1.0) > 0.02 * h * h


def test_constant_linear_and_step_data():
    assert oracle.ppm_face([2.0] * 6) == (2.0, 2.0)
    ql, qr = oracle.ppm_face([0.0, 1.0, 2.0, 3.0, 4.0, 5.0])
    assert ql == pytest.approx(2.5, abs=1e-15) and qr == pytest.approx(2.5, abs=1e-15)
    # a step is not smeared: both zones beside it keep flat parabolas
    assert oracle.ppm_face([0.0, 0.0, 0.0, 1.0, 1.0, 1.0]) == (0.0, 1.0)
    # a local extremum flattens its zone
    ql, qr = oracle.ppm_face([0.0, 0.5, 2.0, 0.4, 0.1, 0.0])
    assert ql == 2.0


def _zone_lr(q, j):
    """(a_L, a_R) of zone j of a longer array (its two face calls)."""
    right = oracle.ppm_face(q[j - 2:j + 4])[0]
    left = oracle.ppm_face(q[j - 3:j + 3])[1]
    return left, right


def test_brute_force_bounds_and_monotone_parabolas():
    rng = np.random.default_rng(11)
    for trial in range(3000):
        kind = trial % 3
        if kind == 0:
            q = rng.normal(size=9)
        elif kind == 1:
            q = np.cumsum(rng.exponential(size=9)) * rng.choice([-1.0, 1.0])   # monotone
        else:
            q = np.sin(rng.uniform(0.2, 2.0) * np.arange(9) + rng.uniform(0, 6))
        ql, qr = oracle.ppm_face(q[1:7])           # the face between q[3] and q[4]
        lo, hi = min(q[3], q[4]), max(q[3], q[4])
        tol = 1e-14 * (1.0 + np.abs(q).max())
        assert lo - tol <= ql <= hi + tol and lo - tol <= qr <= hi + tol, (q, ql, qr)
        a = q[4]
        aL, aR = _zone_lr(q, 4)
        assert (aR - a) * (a - aL) >= -tol * tol, (q, aL, a, aR)
        assert abs(a - 0.5 * (aL + aR)) <= abs(aR - aL) / 6.0 + tol, (q, aL, a, aR)


def _wave_error(n, recon, amp=1e-6):
    G = _flat_grid(n, 1, 1, recon=recon)
    X = _centres(G)[0]
    rho0, u0 = 1.0, 1.0
    p0 = (GAM - 1) * u0
    cs = np.sqrt(GAM * p0 / (rho0 + u0 + p0))
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
    exact = rho0 * (1 + amp * prof(X - cs * t_end))
    return np.abs(Pn[0] - exact).mean() / amp


def test_sound_wave_converges_at_second_order():
    e_ppm = [_wave_error(n, oracle.PPM) for n in (32, 64, 128)]
    e_plm = [_wave_error(n, oracle.PLM) for n in (32, 64, 128)]
    print("sound wave L1 error PPM", e_ppm, "PLM", e_plm)
    assert e_ppm[0] / e_ppm[1] > 3.0 and e_ppm[1] / e_ppm[2] > 3.3, e_ppm
    for a, b in zip(e_ppm, e_plm):
        assert a < 1.6 * b


def test_shock_tube_is_sharper_than_plm():
    from tests import test_oracle_shocktube as T
    from tests.riemann import ExactRiemann

    def l1(n, recon):
        p = oracle.default_params(metric=oracle.MINK_CART, n1=n, n2=1, n3=1, x1min=0.0, x1max=1.0,
                                  x2min=0.0, x2max=1.0, x3min=0.0, x3max=1.0, bc1=oracle.BC_OUTFLOW,
                                  bc2=oracle.BC_OUTFLOW, bc3=oracle.BC_OUTFLOW, gam=T.GAM, recon=recon)
        og = oracle.Grid(p)
        x = (np.arange(n) + 0.5) / n
        P = T._run(og, T._prims_1d(x, T.LEFT, T.RIGHT, T.GAM), T.T_END)
        ex = ExactRiemann(T.LEFT, T.RIGHT, T.GAM)
        rho = np.array([ex.sample((xi - 0.5) / T.T_END)[0] for xi in x])
        return np.abs(P[0, :, 0, 0] - rho).mean()

    e_ppm = [l1(n, oracle.PPM) for n in (100, 200, 400)]
    e_plm = [l1(n, oracle.PLM) for n in (100, 200, 400)]
    print("shock tube L1 PPM", e_ppm, "PLM", e_plm)
    for a, b in zip(e_ppm, e_plm):
        assert a < 0.8 * b
    assert e_ppm[0] / e_ppm[1] > 1.4 and e_ppm[1] / e_ppm[2] > 1.4
