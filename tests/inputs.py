"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module draws random numbers and does plain linear algebra (a Cholesky
factor of a given spatial metric) to place them in a frame.  It holds none of
the method's arithmetic: no metric formula, no conserved variables, no
inversion.  Ranges follow the learned-guess workload of the benchmark
configurations: rho log-uniform in [1e-6, 1], u/rho in [1e-4, 10], Lorentz
factor in [1, 50], sigma = B^2/rho in [1e-3, 100], isotropic directions.
"""
from __future__ import annotations

import numpy as np


def prim_params(n: int, seed: int, rho=(1e-6, 1.0), u_over_rho=(1e-4, 10.0), lorentz=(1.0, 50.0),
                sigma=(1e-3, 100.0)):
    rng = np.random.Generator(np.random.PCG64(seed))

    def logu(lo, hi, size):
        return np.exp(rng.uniform(np.log(lo), np.log(hi), size))

    out = {}
    out["rho"] = logu(*rho, n)
    out["u"] = out["rho"] * logu(*u_over_rho, n)
    # Lorentz factor: log-uniform in (Gamma - 1) over [1e-6, lorentz_max - 1], plus exact 1 for some
    gm1 = logu(1e-6, lorentz[1] - 1.0, n)
    gm1[rng.uniform(size=n) < 0.05] = 0.0
    out["lorentz"] = 1.0 + gm1
    out["sigma"] = logu(*sigma, n)
    v = rng.normal(size=(n, 3))
    out["vdir"] = v / np.linalg.norm(v, axis=1, keepdims=True)
    b = rng.normal(size=(n, 3))
    out["bdir"] = b / np.linalg.norm(b, axis=1, keepdims=True)
    return out


def place_prims(params: dict, gspatial: np.ndarray) -> np.ndarray:
    """Primitives (rho, u, ut^1..3, B^1..3), shape (8, n), for spatial metrics
    gspatial (n, 3, 3): g_ij ut^i ut^j = Gamma^2 - 1 and g_ij B^i B^j = sigma rho."""
    n = gspatial.shape[0]
    L = np.linalg.cholesky(gspatial)
    LT = np.transpose(L, (0, 2, 1))
    ut = np.linalg.solve(LT, params["vdir"][..., None])[..., 0]
    ut *= np.sqrt(params["lorentz"] ** 2 - 1.0)[:, None]
    B = np.linalg.solve(LT, params["bdir"][..., None])[..., 0]
    B *= np.sqrt(params["sigma"] * params["rho"])[:, None]
    P = np.zeros((8, n))
    P[0] = params["rho"]
    P[1] = params["u"]
    P[2:5] = ut.T
    P[5:8] = B.T
    return P


def zone_locations(n: int, n1: int, n2: int, seed: int, near_horizon_frac=0.25, i_h=0):
    """Random active zone locations loc = i*n2 + j, a fraction of them in the
    first four radial zones (near the horizon)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    i = rng.integers(0, n1, n)
    near = rng.uniform(size=n) < near_horizon_frac
    i[near] = rng.integers(i_h, min(i_h + 4, n1), near.sum())
    j = rng.integers(0, n2, n)
    return (i * n2 + j).astype(np.int32)


def perturb_guess(P: np.ndarray, seed: int, rel=0.05) -> np.ndarray:
    """Newton starting point: the true primitives perturbed by a relative amount."""
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    G = P.copy()
    G[0:5] *= 1.0 + rel * rng.uniform(-1.0, 1.0, size=G[0:5].shape)
    return G
