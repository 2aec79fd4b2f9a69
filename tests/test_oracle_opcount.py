"""The operation counter of the oracle's inversion (oracle/opcount.cpp)
pinned by a count made by hand from the source of Section 2.3's Newton
inversion (oracle/con2prim.c), and checked to change nothing in the result.

Hand count, Newton only (methods = 1), started at the exact primitives, so
Newton converges on its first step and takes its one confirming step (2
iterations):
  set-up (B = U_B / sqrt(-g), D, Q_mu, n^mu, Q^mu, n.Q, Qt^2, Qt^i, Bf^i,
          Q.Bf, Bf^2)                     40 add  61 mul   5 div
  start (ut^2, v^2, W)                    12 add  20 mul   1 div
  Newton constants (g1, (Q.B)^2)           1 add   1 mul   1 div
  Newton step (residuals of Eqs. 29-30, Jacobian, 2x2 solve, errors), each
                                          25 add  27 mul   8 div  1 sqrt
  recovery (pressure of Eq. 31, rho, u, ut^i)
                                          10 add   9 mul   8 div  2 sqrt
  total (2 steps): 113 add, 145 mul, 31 div, 4 sqrt = 293 flops.
With the beta switch (methods = 15, magnetised guess): the four-velocity
and b^mu of the guess (66 mul, 45 add, 4 div, 1 sqrt), the gas pressure
(1 add, 1 mul) and the beta test (2 mul): 413 flops.
"""
import numpy as np
import pytest

import oracle

GAM = 4.0 / 3.0


def _zone(magnetised=True):
    og = oracle.Grid(oracle.default_params(n1=32, n2=32, n3=1, gam=GAM, r_out=100.0))
    geom = og.geom_table(0)[10 + oracle.NG, 12 + oracle.NG]
    q = np.array([0.8, 0.3, 0.12, -0.01, 0.05, 0.0, 0.0, 0.0])
    if magnetised:
        q[5:8] = [0.05, 0.004, 0.02]
    U = og.prim2cons(q.reshape(8, 1), np.array([10 * 32 + 12], dtype=np.int32))[:, 0]
    return og, geom, q, U


def test_newton_inversion_count_equals_the_hand_count():
    og, geom, q, U = _zone()
    fl, P, it, n = oracle.count_con2prim(U, geom, q, GAM, methods=1)
    assert fl == oracle.C2P_NR and it == 2
    assert (n["add"], n["mul"], n["div"], n["sqrt"], n["special"]) == (113, 145, 31, 4, 0), n
    assert n["flops"] == 293


def test_beta_switch_adds_the_guess_state():
    og, geom, q, U = _zone()
    fl, P, it, n = oracle.count_con2prim(U, geom, q, GAM, methods=15)
    assert fl == oracle.C2P_NR and it == 2
    assert n["flops"] == 413, n


def test_count_is_linear_in_the_newton_steps():
    # a start away from the root costs more steps; each costs 61 flops
    og, geom, q, U = _zone()
    g = q.copy()
    g[1] *= 1.5
    g[2:5] *= 0.7
    fl, P, it, n = oracle.count_con2prim(U, geom, g, GAM, methods=1)
    assert fl == oracle.C2P_NR and it > 2
    assert n["flops"] == 293 + 61 * (it - 2)


def test_counted_inversion_is_the_oracle_inversion():
    og, geom, q, U = _zone()
    g = q.copy()
    g[1] *= 1.2
    fl, P, it, n = oracle.count_con2prim(U, geom, g, GAM, methods=15)
    loc = np.array([10 * 32 + 12], dtype=np.int32)
    P2, fl2, it2 = og.con2prim(U.reshape(9, 1), loc, g.reshape(8, 1), methods=15)
    assert fl == fl2[0] and it == it2[0]
    assert np.array_equal(P, P2[:, 0])


def test_entropy_inversion_counts_its_power_calls():
    og, geom, q, U = _zone()
    fl, P, it, n = oracle.count_con2prim(U, geom, q, GAM, methods=4)
    assert fl == oracle.C2P_ENTROPY
    assert n["special"] > 0
