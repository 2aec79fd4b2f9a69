"""Michel's transonic spherical accretion onto a Schwarzschild black hole
(Michel 1972), written here from its two conservation laws as a steady
analytic solution for the step tests.

For a polytrope p = K rho^(1+1/n) with T = p/rho, enthalpy h = 1 + (n+1) T and
inflow speed u = -u^r (M = 1), a steady radial flow keeps
  mass:      r^2 rho u            = const,
  Bernoulli: h^2 (1 - 2/r + u^2)  = const.
Eliminating rho, the flow passes smoothly through the sonic radius r_c only if
there u_c^2 = 1/(2 r_c) and the sound speed a^2 = (n+1) T / (n h) equals
u_c^2 / (1 - 3 u_c^2), which fixes T_c.  Elsewhere T solves the Bernoulli
relation on the branch that is subsonic outside r_c and supersonic inside.

The primitives for the step (modified Kerr-Schild, a = 0, r = exp(X1)): u^r is
the same in Schwarzschild and Kerr-Schild coordinates (r is shared), u^t follows
from u.u = -1 in Kerr-Schild, and the primitive velocity is
ut^i = u^i + alpha^2 u^t g^{ti} (Eq. 11 inverted).  On a cylindrified grid
theta depends on X1 too, and u^theta = 0 gives u^2 = -(d theta/dX1 / d theta/dX2) u^1.
"""
from __future__ import annotations

import math

import numpy as np


class Michel:
    def __init__(self, r_c=8.0, n=3.0, rho_c=1e-2):
        self.r_c, self.n = r_c, n
        u2 = 1.0 / (2.0 * r_c)
        a2 = u2 / (1.0 - 3.0 * u2)
        # a^2 = (n+1) T / (n (1 + (n+1) T))  ->  T_c
        self.T_c = a2 * n / ((n + 1.0) * (1.0 - a2 * n))
        self.u_c = math.sqrt(u2)
        self.rho_c = rho_c
        self.K = self.T_c / rho_c ** (1.0 / n)
        self.mdot = r_c ** 2 * rho_c * self.u_c
        self.bern = (1.0 + (n + 1.0) * self.T_c) ** 2 * (1.0 - 2.0 / r_c + u2)

    def rho_of_T(self, T):
        return (T / self.K) ** self.n

    def residual(self, T, r):
        u = self.mdot / (r * r * self.rho_of_T(T))
        return (1.0 + (self.n + 1.0) * T) ** 2 * (1.0 - 2.0 / r + u * u) - self.bern

    def T_of_r(self, r):
        """The transonic branch: at fixed r the Bernoulli residual is positive
        for T -> 0 (u -> infinity) and for large T, with one minimum (the local
        sonic point) between its two roots; take the root above the minimum
        (subsonic) outside r_c and the one below it (supersonic) inside."""
        if abs(r - self.r_c) < 1e-12:
            return self.T_c
        f = lambda lt: self.residual(math.exp(lt), r)
        a, b = math.log(1e-12 * self.T_c), math.log(1e3 * self.T_c)
        for _ in range(200):  # ternary search for the minimum in log T
            m1, m2 = a + (b - a) / 3.0, b - (b - a) / 3.0
            if f(m1) < f(m2):
                b = m2
            else:
                a = m1
        t_min = 0.5 * (a + b)
        lo, hi = (t_min, math.log(1e3 * self.T_c)) if r > self.r_c else (math.log(1e-12 * self.T_c), t_min)
        f_lo = f(lo)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            f_mid = f(mid)
            if (f_mid > 0) == (f_lo > 0):
                lo, f_lo = mid, f_mid
            else:
                hi = mid
        return math.exp(0.5 * (lo + hi))

    def state(self, r):
        T = self.T_of_r(r)
        rho = self.rho_of_T(T)
        u = self.mdot / (r * r * rho)
        return rho, T, u


def michel_prims(og, mic: Michel, gam: float):
    """Primitives (8, n1, n2, n3) of the Michel flow on an oracle grid (a = 0,
    MKS with r = exp(X1)); gam = 1 + 1/n."""
    n1, n2, n3 = og.shape
    tab = og.geom_table(0)
    NG = og.ng
    P = np.zeros((8, n1, n2, n3))
    for i in range(n1):
        X1 = og.x1in + (i + 0.5) * og.dx[0]
        r = og.r_of_x1(X1)
        rho, T, u = mic.state(r)
        drdx = r
        for j in range(n2):
            g = tab[i + NG, j + NG]
            gcov = g[:16].reshape(4, 4)
            gcon = g[16:32].reshape(4, 4)
            alpha = g[33]
            u1 = -u / drdx
            _, th1, th2 = og.theta_at(X1, og.x2in + (og.p.j0 + j + 0.5) * og.dx[1])
            u2 = -th1 * u1 / th2
            # g_tt (u^t)^2 + 2 (g_t1 u^1 + g_t2 u^2) u^t + g_ij u^i u^j = -1;
            # the future root in the form that stays finite where g_tt
            # changes sign at r = 2
            A = gcov[0, 0]
            B = 2.0 * (gcov[0, 1] * u1 + gcov[0, 2] * u2)
            C = (gcov[1, 1] * u1 * u1 + 2.0 * gcov[1, 2] * u1 * u2 + gcov[2, 2] * u2 * u2) + 1.0
            disc = B * B - 4.0 * A * C
            ut = 2.0 * C / (-B + math.sqrt(disc))
            P[0, i, j, :] = rho
            P[1, i, j, :] = rho * T / (gam - 1.0)
            P[2, i, j, :] = u1 + alpha * alpha * ut * gcon[0, 1]
            P[3, i, j, :] = u2 + alpha * alpha * ut * gcon[0, 2]
    return P
