"""Helpers shared by the GPU parity tests: matching oracle / GPU grids and the
per-field error metric.

Per-field parity metric (FP64 path), for a state array x[f, ...]:
  - positive-definite fields (rho, u; U_rho, -U_E, U_S) -- pointwise relative
    error max_z |x_gpu - x_orc| / |x_orc|;
  - signed fields (velocities, B, momenta) -- max-norm relative error
    max_z |x_gpu - x_orc| / max_z |x_orc|, because their values can be far
    smaller than the terms that produce them (e.g. u^theta of a torus in
    equilibrium, or B^3 grown from zero by shear), so a pointwise ratio
    measures that cancellation rather than the implementation.
Target: 1e-10 per step.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def have_gpu():
    return torch.cuda.is_available()


def gpu_mod():
    from paper_2205_02484_gb300 import build, grmhd
    build.build()
    grmhd.load()
    return grmhd


def make_pair(n1, n2, n3, gam=13.0 / 9.0, a=0.9375, r_out=40.0, precision=0, metric=0, riemann=0,
              stream=True, phys=None, **box):
    """Oracle grid and GPU context with identical parameters (phys: solver
    and limit parameters set on both sides, e.g. nr_maxit)."""
    G = gpu_mod()
    phys = dict(phys or {})
    kw = dict(n1=n1, n2=n2, n3=n3, gam=gam, a=a, r_out=r_out, metric=metric, riemann=riemann)
    kw.update(box)
    kw.update(phys)
    op = oracle.default_params(**kw)
    og = oracle.Grid(op)
    gkw = dict(r_out=r_out, precision=precision, metric=metric, riemann=riemann, a=a)
    gkw.update(box)
    gp = G.default_grid(n1, n2, n3, **gkw)
    if stream:
        gp.stream = torch.cuda.current_stream().cuda_stream
    ctx = G.init_grid(gp, G.default_phys(gam=gam, **phys))
    G.set_metric(ctx, a, metric)
    return og, ctx


POS_P = (0, 1)        # rho, u
POS_U = (0, 1, 8)     # U_rho, U_E (negative definite), U_S


def field_err(x_gpu, x_orc, positive=None):
    """per-field error: pointwise relative for positive-definite fields,
    max-norm relative for the others"""
    if positive is None:
        positive = POS_P if x_orc.shape[0] == 8 else POS_U
    out = []
    for f in range(x_orc.shape[0]):
        a, b = x_gpu[f], x_orc[f]
        scale = np.abs(b).max()
        if scale == 0.0:
            out.append(np.abs(a).max())
        elif f in positive:
            out.append((np.abs(a - b) / np.abs(b)).max())
        else:
            out.append(np.abs(a - b).max() / scale)
    return np.array(out)


def pointwise_err(x_gpu, x_orc):
    """The per-field metric err_f = max_z |x_gpu - x_orc| / (|x_orc| +
    1e-12 max_z |x_orc|), pointwise for every field (reported beside
    field_err, whose signed fields use the max-norm)."""
    out = []
    for f in range(x_orc.shape[0]):
        a, b = x_gpu[f], x_orc[f]
        den = np.abs(b) + 1e-12 * np.abs(b).max() + 1e-300
        out.append((np.abs(a - b) / den).max())
    return np.array(out)
