"""Flat-space shock tubes (Minkowski metric, Cartesian box): the oracle's step
converges in L1 to the exact relativistic hydrodynamic Riemann solution, and a
magnetised tube and its mirror image evolve into mirror images.  The initial
states are chosen here (synthetic); no external benchmark states are used."""
import math

import numpy as np
import pytest

import oracle
from tests.riemann import ExactRiemann, State

GAM = 4.0 / 3.0
LEFT = State(5.0, 4.0, 0.2)
RIGHT = State(1.0, 0.1, -0.1)
T_END = 0.3


def _tube(n, bc=oracle.BC_OUTFLOW, riemann=oracle.LLF):
    p = oracle.default_params(metric=oracle.MINK_CART, n1=n, n2=1, n3=1, x1min=0.0, x1max=1.0,
                              x2min=0.0, x2max=1.0, x3min=0.0, x3max=1.0, bc1=bc, bc2=bc, bc3=bc, gam=GAM,
                              riemann=riemann)
    return oracle.Grid(p)


def _prims_1d(x, left, right, gam, B=None):
    P = np.zeros((8, x.size, 1, 1))
    for k, (st, sel) in enumerate(((left, x < 0.5), (right, x >= 0.5))):
        W = 1.0 / math.sqrt(1.0 - st.v ** 2)
        P[0, sel] = st.rho
        P[1, sel] = st.p / (gam - 1.0)
        P[2, sel] = W * st.v
    if B is not None:
        for c in range(3):
            P[5 + c, x < 0.5] = B[0][c]
            P[5 + c, x >= 0.5] = B[1][c]
    return P


def _run(og, P, t_end):
    U = og.prim2cons(P.reshape(8, -1), np.zeros(P[0].size, dtype=np.int32)).reshape((9,) + P.shape[1:])
    og.set_state(P, U, 0.0, 0.0)
    og.set_dt(og.initial_dt())
    while True:
        _, _, t, dt = og.get_state()
        if t >= t_end - 1e-14:
            break
        if t + dt > t_end:
            og.set_dt(t_end - t)
        assert og.step() == 0
    return og.get_state()[0]


def test_exact_solution_satisfies_the_jump_conditions():
    ex = ExactRiemann(LEFT, RIGHT, GAM)
    # pressure and velocity are continuous across the contact
    assert ex.wl[1] == ex.wr[1] and abs(ex.wl[2] - ex.wr[2]) < 1e-12
    for st, w in ((LEFT, ex.wl), (RIGHT, ex.wr)):
        rho_b, p_b, v_b, V = w
        if p_b > st.p:  # shock: F(U_b) - F(U_a) = V (U_b - U_a)
            Ua, Fa = ex.cons_flux(st.rho, st.p, st.v)
            Ub, Fb = ex.cons_flux(rho_b, p_b, v_b)
            for c in range(3):
                assert Fb[c] - Fa[c] == pytest.approx(V * (Ub[c] - Ua[c]), rel=1e-9, abs=1e-12)
        else:  # rarefaction: isentropic, the invariant of the other family conserved
            assert p_b / rho_b ** GAM == pytest.approx(st.p / st.rho ** GAM, rel=1e-12)
    # this pair makes a left rarefaction and a right shock
    assert ex.wl[1] < LEFT.p and ex.wr[1] > RIGHT.p
    # the sampled solution joins the end states
    assert ex.sample(-0.99) == (LEFT.rho, LEFT.p, LEFT.v)
    assert ex.sample(0.99) == (RIGHT.rho, RIGHT.p, RIGHT.v)


def _l1_error(n, riemann=oracle.LLF):
    og = _tube(n, riemann=riemann)
    x = (np.arange(n) + 0.5) / n
    P = _run(og, _prims_1d(x, LEFT, RIGHT, GAM), T_END)
    ex = ExactRiemann(LEFT, RIGHT, GAM)
    rho_ex = np.array([ex.sample((xi - 0.5) / T_END)[0] for xi in x])
    return np.abs(P[0, :, 0, 0] - rho_ex).mean()


@pytest.mark.parametrize("riemann", [oracle.LLF, oracle.HLL])
def test_tube_converges_to_the_exact_solution(riemann):
    e = [_l1_error(n, riemann) for n in (100, 200, 400)]
    # shocks and the contact limit L1 convergence to about first order; the
    # shocked shell between the contact and the shock is 0.04 wide at t = 0.3
    assert e[0] / e[1] > 1.5 and e[1] / e[2] > 1.5, e
    assert e[2] < 0.04


def test_hll_resolves_the_tube_better_than_llf():
    # HLL (Eq. 21) uses the one-sided signal speeds, LLF (Eq. 18) the largest
    # speed on both sides, so HLL adds less dissipation on this tube
    for n in (100, 200):
        assert _l1_error(n, oracle.HLL) < 0.9 * _l1_error(n, oracle.LLF)


def test_magnetised_tube_mirror_symmetry():
    n = 96
    x = (np.arange(n) + 0.5) / n
    B = ((0.5, 1.0, 0.3), (0.5, -0.7, 0.2))
    P = _prims_1d(x, LEFT, RIGHT, GAM, B)
    # mirror image x -> 1 - x: states swapped, v_x and B_x reversed (the
    # equations are unchanged under x -> -x together with B -> -B)
    M = P[:, ::-1].copy()
    M[2] *= -1.0
    M[6:8] *= -1.0
    Pa = _run(_tube(n), P, 0.25)
    Pb = _run(_tube(n), M, 0.25)
    Mb = Pb[:, ::-1].copy()
    Mb[2] *= -1.0
    Mb[6:8] *= -1.0
    for f in range(8):
        scale = np.abs(Pa[f]).max() + 1e-300
        assert np.abs(Mb[f] - Pa[f]).max() <= 1e-12 * scale, f
