"""Pins of the oracle's Riemann fluxes (Eqs. 18, 21) and of the limits of
Section 2.4 (magnetisation ceilings by mass added in the normal frame, the
Lorentz-factor cap).

Every expected value is built here from closed forms, not from the oracle's
own routines: the flat-space conserved vector and flux of a moving perfect
fluid, relativistic velocity addition for the signal speeds, the conserved
vector of matter at rest in the normal (ZAMO) frame, and the normalisation
Gamma^2 = 1 + g_ij ut^i ut^j of the modified velocity (Eq. 11).  A swapped
c_max / c_min, a wrong sign of the dissipative term, a ceiling that adds
moving matter or a cap that turns the velocity would each fail one of them.
"""
import math

import numpy as np
import pytest

import oracle

GAM = 4.0 / 3.0


# ----------------------------------------------------------- flat-space fluxes

def _flat_grid(riemann):
    p = oracle.default_params(metric=oracle.MINK_CART, n1=8, n2=1, n3=1, x1min=0.0, x1max=1.0,
                              x2min=0.0, x2max=1.0, x3min=0.0, x3max=1.0, bc1=oracle.BC_OUTFLOW,
                              bc2=oracle.BC_OUTFLOW, bc3=oracle.BC_PERIODIC, gam=GAM, riemann=riemann)
    return oracle.Grid(p)


def _hydro(rho, p, v):
    """Primitives (Eq. 11) of a flat-space fluid moving along x with speed v."""
    W = 1.0 / math.sqrt(1.0 - v * v)
    return np.array([rho, p / (GAM - 1.0), W * v, 0, 0, 0, 0, 0], dtype=float)


def _UF(rho, p, v):
    """Closed-form conserved vector and x-flux of a flat-space perfect fluid
    moving along x: T^mu_nu = w u^mu u_nu + p delta, u^mu = W (1, v, 0, 0),
    u_mu = W (-1, v, 0, 0), w = rho + u + p, S = p / rho^(gam-1)."""
    W = 1.0 / math.sqrt(1.0 - v * v)
    w = rho + p / (GAM - 1.0) + p
    S = p / rho ** (GAM - 1.0)
    U = np.array([rho * W, -w * W * W + p, w * W * W * v, 0, 0, 0, 0, 0, S * W])
    F = np.array([rho * W * v, -w * W * W * v, w * W * W * v * v + p, 0, 0, 0, 0, 0, S * W * v])
    return U, F


def _speeds(rho, p, v):
    """Signal speeds (v +- c_s) / (1 +- v c_s) of a flat-space fluid along its motion."""
    cs = math.sqrt(GAM * p / (rho + p / (GAM - 1.0) + p))
    return (v + cs) / (1.0 + v * cs), (v - cs) / (1.0 - v * cs)


def _face(G, L, R):
    """Riemann flux of the X1 face between two uniform states (flat slopes)."""
    q4 = np.stack([L, L, R, R])
    F, cw = G.face_flux_at(0, 4, 0, q4)
    return F, cw


CASES = [((1.0, 1.0, 0.0), (0.125, 0.1, 0.0)),   # Sod-like, both at rest
         ((5.0, 4.0, 0.2), (1.0, 0.1, -0.1)),     # opposite motions
         ((0.3, 0.02, 0.5), (2.0, 3.0, -0.6))]    # fast, hot right state


@pytest.mark.parametrize("left,right", CASES)
def test_hll_and_llf_against_closed_forms(left, right):
    Ul, Fl = _UF(*left)
    Ur, Fr = _UF(*right)
    c1l, c2l = _speeds(*left)
    c1r, c2r = _speeds(*right)
    cmax = max(0.0, c1l, c1r)
    cmin = max(0.0, -c2l, -c2r)
    hll = (cmax * Fl + cmin * Fr - cmax * cmin * (Ur - Ul)) / (cmax + cmin)
    cw = max(cmax, cmin)
    llf = 0.5 * (Fl + Fr - cw * (Ur - Ul))
    scale = np.abs(Fl).max() + np.abs(Fr).max() + cw * (np.abs(Ul).max() + np.abs(Ur).max())
    for riemann, ref in ((oracle.HLL, hll), (oracle.LLF, llf)):
        F, c = _face(_flat_grid(riemann), _hydro(*left), _hydro(*right))
        assert abs(c - cw) < 1e-14
        assert np.abs(F - ref).max() < 1e-13 * scale, (riemann, F, ref)


@pytest.mark.parametrize("v", [0.9, -0.9])
def test_hll_is_upwind_for_supersonic_flow(v):
    # both states move faster than sound in one direction: every signal speed
    # has that sign, so one of c_max, c_min is 0 and HLL is the upwind flux
    left, right = (1.0, 0.1, v), (0.5, 0.05, v)
    for st in (left, right):
        c1, c2 = _speeds(*st)
        assert c1 * c2 > 0 and c1 * v > 0
    F, _ = _face(_flat_grid(oracle.HLL), _hydro(*left), _hydro(*right))
    _, Fl = _UF(*left)
    _, Fr = _UF(*right)
    up = Fl if v > 0 else Fr
    assert np.abs(F - up).max() < 1e-14 * np.abs(up).max()
    # LLF keeps its dissipation and is not the upwind flux
    G = _flat_grid(oracle.LLF)
    Fll, _ = _face(G, _hydro(*left), _hydro(*right))
    assert np.abs(Fll - up).max() > 1e-3 * np.abs(up).max()


def test_hll_equals_llf_when_the_signal_speeds_are_symmetric():
    # two states at rest with the same sound speed (rho, p scaled together):
    # c_max = c_min, and Eq. 21 reduces to Eq. 18
    L, R = _hydro(1.0, 0.6, 0.0), _hydro(0.25, 0.15, 0.0)
    Fh, ch = _face(_flat_grid(oracle.HLL), L, R)
    Fl, cl = _face(_flat_grid(oracle.LLF), L, R)
    assert ch == cl
    assert np.abs(Fh - Fl).max() < 1e-15 * np.abs(Fl).max()


@pytest.mark.parametrize("riemann", [oracle.HLL, oracle.LLF])
def test_flux_consistency(riemann):
    # F(q, q) = F(q) for a moving, magnetised state
    q = np.array([0.8, 0.4, 0.3, -0.2, 0.1, 0.5, 0.2, -0.4])
    F, _ = _face(_flat_grid(riemann), q, q)
    g = oracle.geom_from(np.diag([-1.0, 1.0, 1.0, 1.0]))
    ref = oracle.prim_to_F(q, g, GAM, 1)
    assert np.abs(F - ref).max() < 1e-15 * np.abs(ref).max()


# ------------------------------------------------ Kerr zone helpers (numpy)

def _kerr_grid(n1=48, n2=48, a=0.9375, **kw):
    p = oracle.default_params(n1=n1, n2=n2, n3=1, a=a, r_out=100.0, gam=GAM, **kw)
    return oracle.Grid(p)


def _zone_metric(G, i, j):
    row = G.geom_table(0)[i + oracle.NG, j + oracle.NG]
    return row[:16].reshape(4, 4), row[16:32].reshape(4, 4), row[32], row[33]


def _fluid(gcov, gcon, q):
    """u^mu, u_mu, b^mu, b_mu, b^2 and Gamma of primitives q from their
    definitions (Eq. 11 and Section 2.1)."""
    alpha = 1.0 / math.sqrt(-gcon[0, 0])
    ut = q[2:5]
    gam = math.sqrt(1.0 + ut @ gcov[1:, 1:] @ ut)
    ucon = np.empty(4)
    ucon[0] = gam / alpha
    ucon[1:] = ut - gam * alpha * gcon[0, 1:]
    ucov = gcov @ ucon
    B = q[5:8]
    bcon = np.empty(4)
    bcon[0] = B @ ucov[1:]
    bcon[1:] = (B + bcon[0] * ucon[1:]) / ucon[0]
    bsq = bcon @ gcov @ bcon
    return ucon, ucov, bsq, gam, alpha


def _state(G, i, j, rho, u, ut, B):
    q = np.array([rho, u, *ut, *B], dtype=float)
    loc = np.array([(i + 0) * G.p.n2 + j], dtype=np.int32)  # active zone index (k = 0)
    U = G.prim2cons(q.reshape(8, 1), loc)[:, 0]
    return q, U, loc


def _rest_frame_U(gdet, alpha, drho, du):
    """Conserved vector of matter at rest in the normal frame: u^mu = n^mu,
    u_mu = (-alpha, 0, 0, 0), so sqrt(-g) rho u^t = sqrt(-g) drho / alpha,
    sqrt(-g) T^t_t = -sqrt(-g) (drho + du), sqrt(-g) T^t_i = 0."""
    return gdet * np.array([drho / alpha, -(drho + du), 0.0, 0.0, 0.0])


# ------------------------------------------------------------- ceilings

@pytest.mark.parametrize("zone", [(10, 12), (30, 24), (6, 40)])
def test_ceiling_adds_matter_at_rest_in_the_normal_frame(zone):
    i, j = zone
    G = _kerr_grid()
    gcov, gcon, gdet, alpha = _zone_metric(G, i, j)
    # a moving, strongly magnetised zone: b^2/rho ~ 4 x 50, b^2/u ~ 2 x 2500
    q0 = np.array([1.0, 1.0, 0.3, -0.02, 0.05, 0.0, 0.0, 0.0])
    q0[5:8] = [0.2, 0.01, 0.1]
    _, _, bsq1, _, _ = _fluid(gcov, gcon, q0)
    q0[5:8] *= math.sqrt(4 * 50 / bsq1)            # b^2 = 200 at rho = 1
    q0[1] = q0[0] * 50 * 4 / (2 * 2500)            # b^2 / u = 5000
    q, U, _ = _state(G, i, j, q0[0], q0[1], q0[2:5], q0[5:8])
    _, _, bsq, _, _ = _fluid(gcov, gcon, q)
    drho, du = bsq / 50.0 - q[0], bsq / 2500.0 - q[1]
    assert drho > 0 and du > 0
    qn, mod, nceil, ncap = G.post_inversion(i, j, q, U)
    assert mod == 1 and nceil == 1 and ncap == 0
    # the new primitives are the inversion of U + dU, dU that of matter at rest
    # in the normal frame with the missing rho and u; B is untouched
    loc = np.array([i * G.p.n2 + j], dtype=np.int32)
    Un = G.prim2cons(qn.reshape(8, 1), loc)[:, 0]
    dU = _rest_frame_U(gdet, alpha, drho, du)
    scale = np.abs(U[:5]).max() + np.abs(dU).max()
    assert np.abs((Un[:5] - U[:5]) - dU).max() < 1e-9 * scale, (Un[:5] - U[:5], dU)
    assert np.array_equal(qn[5:8], q[5:8])
    assert np.array_equal(Un[5:8], U[5:8])


def test_ceiling_of_a_fluid_at_rest_reaches_the_limits_exactly():
    # ut = 0 (at rest in the normal frame): the added matter keeps it at rest,
    # b^2 does not change, and rho, u land on b^2/50 and b^2/2500
    i, j = 20, 17
    G = _kerr_grid()
    gcov, gcon, gdet, alpha = _zone_metric(G, i, j)
    q, U, _ = _state(G, i, j, 1e-3, 1e-6, [0.0, 0.0, 0.0], [0.05, 0.002, 0.03])
    _, _, bsq, _, _ = _fluid(gcov, gcon, q)
    assert bsq / q[0] > 50 and bsq / q[1] > 2500
    qn, mod, nceil, _ = G.post_inversion(i, j, q, U)
    assert nceil == 1
    _, _, bsq_n, gam_n, _ = _fluid(gcov, gcon, qn)
    assert abs(gam_n - 1.0) < 1e-12
    assert abs(bsq_n / qn[0] - 50.0) < 1e-9 * 50.0
    assert abs(bsq_n / qn[1] - 2500.0) < 1e-9 * 2500.0


def test_no_ceiling_below_the_limits():
    i, j = 20, 17
    G = _kerr_grid()
    q, U, _ = _state(G, i, j, 1.0, 0.5, [0.1, 0.0, 0.2], [0.05, 0.002, 0.03])
    qn, mod, nceil, ncap = G.post_inversion(i, j, q, U)
    assert (mod, nceil, ncap) == (0, 0, 0)
    assert np.array_equal(qn, q)


# ---------------------------------------------------------- Lorentz cap

@pytest.mark.parametrize("lorentz", [80.0, 400.0])
def test_lorentz_cap_rescales_the_velocity_to_gamma_max(lorentz):
    i, j = 14, 30
    G = _kerr_grid()
    gcov, gcon, _, _ = _zone_metric(G, i, j)
    d = np.array([0.7, -0.05, 0.3])
    d /= math.sqrt(d @ gcov[1:, 1:] @ d)           # unit length in the spatial metric
    ut = d * math.sqrt(lorentz ** 2 - 1.0)
    q, U, _ = _state(G, i, j, 1.0, 0.1, ut, [0.0, 0.0, 0.0])
    assert abs(_fluid(gcov, gcon, q)[3] - lorentz) < 1e-9 * lorentz
    qn, mod, nceil, ncap = G.post_inversion(i, j, q, U)
    assert mod == 1 and nceil == 0 and ncap == 1
    gam = _fluid(gcov, gcon, qn)[3]
    assert abs(gam - 50.0) < 1e-12 * 50.0
    # the direction of ut is kept: ut' = f ut with f > 0
    f = qn[2:5] / q[2:5]
    assert np.all(f > 0) and np.ptp(f) < 1e-14
    assert np.array_equal(qn[[0, 1, 5, 6, 7]], q[[0, 1, 5, 6, 7]])


def test_lorentz_cap_leaves_slower_flow_alone():
    i, j = 14, 30
    G = _kerr_grid()
    gcov, gcon, _, _ = _zone_metric(G, i, j)
    d = np.array([0.7, -0.05, 0.3])
    d /= math.sqrt(d @ gcov[1:, 1:] @ d)
    q, U, _ = _state(G, i, j, 1.0, 0.1, d * math.sqrt(49.9 ** 2 - 1.0), [0.0, 0.0, 0.0])
    qn, mod, _, ncap = G.post_inversion(i, j, q, U)
    assert (mod, ncap) == (0, 0) and np.array_equal(qn, q)
