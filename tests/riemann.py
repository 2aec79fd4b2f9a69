"""Exact solution of the special-relativistic hydrodynamic Riemann problem
(ideal gas, flow along x only), for the shock-tube pins.

Written from the conservation laws rather than from a published listing:
- across a shock, the Rankine-Hugoniot conditions F(U_b) - F(U_a) =
  V_s (U_b - U_a) of the relativistic Euler equations (mass D = rho W,
  momentum S = rho h W^2 v, energy tau = rho h W^2 - p - D) are solved for the
  state behind a shock of given pressure, through the Taub adiabat
  [h^2] = (h_b/rho_b + h_a/rho_a)(p_b - p_a) and the invariant mass flux
  j^2 = -[p]/[h/rho];
- across a rarefaction, the Riemann invariant of the other family,
  atanh(v) +- int c_s d(rho)/rho along the isentrope p = K rho^gam, is
  constant (the sign by the wave's direction);
- the star pressure makes the velocities behind the two waves equal.
The solution depends on x and t only through xi = (x - x0)/t.
"""
from __future__ import annotations

import math
import warnings

from scipy.integrate import IntegrationWarning, quad


class State:
    def __init__(self, rho, p, v):
        self.rho, self.p, self.v = float(rho), float(p), float(v)


def _bisect(f, lo, hi, n=200):
    flo = f(lo)
    for _ in range(n):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


class ExactRiemann:
    def __init__(self, L: State, R: State, gam: float):
        self.L, self.R, self.gam = L, R, gam
        self.g = gam / (gam - 1.0)
        lo = 1e-12 * min(L.p, R.p)
        hi = 1e3 * max(L.p, R.p)
        dv = lambda lp: self._behind(L, math.exp(lp), -1)[2] - self._behind(R, math.exp(lp), +1)[2]
        self.p_star = math.exp(_bisect(dv, math.log(lo), math.log(hi)))
        self.wl = self._behind(L, self.p_star, -1)
        self.wr = self._behind(R, self.p_star, +1)
        self.v_star = 0.5 * (self.wl[2] + self.wr[2])

    # ---- thermodynamics
    def h(self, rho, p):
        return 1.0 + self.g * p / rho

    def cs(self, rho, p):
        return math.sqrt(self.gam * p / (rho * self.h(rho, p)))

    # ---- the state behind a wave of pressure p facing direction s (-1 left, +1 right)
    def _behind(self, a: State, p, s):
        """(rho_b, p, v_b, wave speed) -- shock if p > p_a, else rarefaction
        (wave speed = the tail of the fan)."""
        if p > a.p:
            rho_b, V = self._shock(a, p, s)
            return rho_b, p, self._v_behind_shock(a, rho_b, V), V
        rho_b = a.rho * (p / a.p) ** (1.0 / self.gam)
        dI = self._int_cs(a, a.rho, rho_b)
        # left fan (s = -1): atanh v + I constant; right fan (s = +1): atanh v - I constant
        v_b = math.tanh(math.atanh(a.v) + s * dI)
        c_b = self.cs(rho_b, p)
        tail = (v_b + s * c_b) / (1.0 + s * v_b * c_b)
        return rho_b, p, v_b, tail

    def _int_cs(self, a: State, r0, r1):
        K = a.p / a.rho ** self.gam
        with warnings.catch_warnings():
            # a smooth integrand; quad only reports that it cannot beat rounding
            warnings.simplefilter("ignore", IntegrationWarning)
            return quad(lambda r: self.cs(r, K * r ** self.gam) / r, r0, r1, epsabs=1e-14, epsrel=1e-10,
                        limit=200)[0]

    def _shock(self, a: State, pb, s):
        """rho behind and shock speed for a shock of pressure pb into state a."""
        g, ha = self.g, self.h(a.rho, a.p)
        dp = pb - a.p
        # Taub adiabat in x = 1/rho_b:  (1 + g pb x)^2 - ha^2 = ((1 + g pb x) x + ha/rho_a) dp
        A = g * g * pb * pb - g * pb * dp
        B = 2.0 * g * pb - dp
        C = 1.0 - ha * ha - dp * ha / a.rho
        disc = B * B - 4.0 * A * C
        roots = [(-B + sgn * math.sqrt(disc)) / (2.0 * A) for sgn in (1.0, -1.0)]
        x = max(r for r in roots if r > 0.0)
        rho_b = 1.0 / x
        hb = self.h(rho_b, pb)
        j2 = dp / (ha / a.rho - hb / rho_b)
        Wa = 1.0 / math.sqrt(1.0 - a.v * a.v)
        # mass flux through the shock rho_a W_a W_s (V - v_a) = s |j|
        f = lambda V: a.rho * Wa * (V - a.v) / math.sqrt(1.0 - V * V) - s * math.sqrt(j2)
        V = _bisect(f, -1.0 + 1e-15, 1.0 - 1e-15)
        return rho_b, V

    def _v_behind_shock(self, a: State, rho_b, V):
        Wa = 1.0 / math.sqrt(1.0 - a.v * a.v)
        m = a.rho * Wa * (V - a.v)  # rho W (V - v) is continuous
        f = lambda v: rho_b * (V - v) / math.sqrt(1.0 - v * v) - m
        return _bisect(f, -1.0 + 1e-15, 1.0 - 1e-15)

    # ---- sampling
    def sample(self, xi):
        """(rho, p, v) at xi = (x - x0)/t."""
        L, R = self.L, self.R
        if xi < self.v_star:
            a, s, w = L, -1, self.wl
        else:
            a, s, w = R, +1, self.wr
        rho_b, p_b, v_b, tail = w
        if p_b > a.p:  # shock
            V = tail
            ahead = xi < V if s < 0 else xi > V
            return (a.rho, a.p, a.v) if ahead else (rho_b, p_b, v_b)
        ca = self.cs(a.rho, a.p)
        head = (a.v + s * ca) / (1.0 + s * a.v * ca)
        if (s < 0 and xi <= head) or (s > 0 and xi >= head):
            return a.rho, a.p, a.v
        if (s < 0 and xi >= tail) or (s > 0 and xi <= tail):
            return rho_b, p_b, v_b
        # inside the fan: the characteristic (v + s c)/(1 + s v c) = xi through the state on the invariant
        K = a.p / a.rho ** self.gam

        def fan_xi(rho):
            p = K * rho ** self.gam
            v = math.tanh(math.atanh(a.v) + s * self._int_cs(a, a.rho, rho))
            c = self.cs(rho, p)
            return (v + s * c) / (1.0 + s * v * c) - xi

        rho = _bisect(fan_xi, rho_b, a.rho, n=80)
        p = K * rho ** self.gam
        v = math.tanh(math.atanh(a.v) + s * self._int_cs(a, a.rho, rho))
        return rho, p, v

    # ---- conserved variables and fluxes (for the jump-condition check)
    def cons_flux(self, rho, p, v):
        W = 1.0 / math.sqrt(1.0 - v * v)
        h = self.h(rho, p)
        D, S, E = rho * W, rho * h * W * W * v, rho * h * W * W - p
        return (D, S, E), (D * v, S * v + p, S)
