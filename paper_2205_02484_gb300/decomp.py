"""Phi-slab decomposition of the step: the slab layout of the paper's
multi-GPU runs (Section 3), split along phi, over contexts whose X3 ghosts
are external (BC_EXTERNAL).

One step of the decomposed grid:
  1. every slab runs the predictor (Eq. 25) and reports its per-direction
     CFL minima (the terms of Eq. 27);
  2. the NG = 2 X3 ghost planes of P-hat are exchanged with the phi
     neighbours (periodic in phi);
  3. every slab runs the corrector (Eq. 26);
  4. the ghost planes of P are exchanged;
  5. the minima are reduced over slabs by a minimum, and every slab advances
     t and sets the next dt from Eq. 27.
The metric does not depend on phi, each slab's ghost planes hold exactly the
values the undecomposed grid would read there (taken after the neighbour's
own X1/X2 boundary fill), and a minimum is exact, so the decomposed step
equals the undecomposed one bit for bit -- provided a slab's dX3 equals the
whole grid's, which slab_grid guarantees for power-of-two slab widths.

Two drivers, both over any object with the SlabEngine methods:
  SlabRing -- all slabs on one device and one stream; the exchange is a pack
              and an unpack through device buffers;
  SlabRank -- one slab per process; the exchange is point-to-point sends of
              torch.distributed, the dt reduction a MIN all-reduce.
CtxSlab is the engine over the CUDA library.
"""
from __future__ import annotations

import contextlib
import math

import torch

from . import grmhd as G

NG = 2


def slab_grid(base: G.GridParams, R: int) -> G.GridParams:
    """Grid parameters of one of R phi slabs of `base` (n3 / R zones, X3
    ghosts external).  The step uses a slab's phi position nowhere (the
    metric is axisymmetric, the Minkowski box uniform), only dX3, so every
    slab spans [0, (n3 / R) dX3)."""
    if R < 1 or base.n3 % R:
        raise ValueError(f"n3 = {base.n3} does not split into {R} slabs")
    n3 = base.n3 // R
    if n3 < NG:
        raise ValueError(f"slabs of {n3} < {NG} phi zones")
    h = 2.0 * math.pi / base.n3 if base.metric == G.KERR_MKS else (base.x3max - base.x3min) / base.n3
    g = G.GridParams.from_buffer_copy(base)
    g.n3, g.bc3, g.x3min, g.x3max = n3, G.BC_EXTERNAL, 0.0, n3 * h
    return g


def split_phi(x, R: int, r: int):
    """Slab r's part of a (fields, n1, n2, n3) array (numpy or torch), contiguous."""
    n3 = x.shape[3] // R
    part = x[..., r * n3:(r + 1) * n3]
    return part.contiguous() if isinstance(x, torch.Tensor) else part.copy(order="C")


class CtxSlab:
    """SlabEngine over one grmhd context with bc3 = BC_EXTERNAL.  Every call
    is asynchronous on the context's stream (`stream`)."""

    def __init__(self, ctx: G.Context, stream: torch.cuda.Stream):
        if ctx.grid.bc3 != G.BC_EXTERNAL:
            raise ValueError("a slab context needs bc3 = BC_EXTERNAL")
        self.ctx = ctx
        self.stream = stream
        self.device = torch.device("cuda", ctx.grid.device)
        self.dtype = torch.float64 if ctx.grid.precision == G.FP64 else torch.float32
        self.plane_numel = G.x3_plane_bytes(ctx) // (8 if self.dtype == torch.float64 else 4)

    @classmethod
    def create(cls, grid: G.GridParams, phys: G.PhysParams, a: float, stream: torch.cuda.Stream):
        g = G.GridParams.from_buffer_copy(grid)
        g.stream = stream.cuda_stream
        ctx = G.init_grid(g, phys)
        G.set_metric(ctx, a, g.metric)
        return cls(ctx, stream)

    def set_state(self, P, U, t, dt):
        G.set_state(self.ctx, P, U, t, dt)

    def get_state(self):
        return G.get_state(self.ctx)

    def diagnostics(self):
        return G.diagnostics(self.ctx)

    def barycentric_sums(self, r_bar_max):
        _, den, num = G.barycentric_radius(self.ctx, r_bar_max)
        return num, den

    def stage(self, st):
        G.stage(self.ctx, st)

    def dtd(self, out, accumulate=False):
        G.step_dtd(self.ctx, out, accumulate)

    def finish(self, dtd):
        G.finish_step(self.ctx, dtd)

    def pack(self, which, side, buf):
        G.x3_pack(self.ctx, which, side, buf)

    def unpack(self, which, side, buf):
        G.x3_unpack(self.ctx, which, side, buf)

    def close(self):
        self.ctx.close()


_SUMMED = ("mdot", "phib", "edot", "ldot", "nr_iters", "n_nr", "n_brent", "n_entropy", "n_entropy_beta",
           "n_fail", "n_floor", "n_ceil", "n_gcap", "n_fixed", "fix_sweeps")


def combine_diagnostics(parts):
    """Whole-grid horizon diagnostics (Eqs. 38-42) from the slabs' own: the
    shell integrals and the counters add up, the normalised flux is formed
    from the sums, div B is the largest over the slabs (each checks the
    corners inside it).  t, dt and the step count are the slabs' common
    values; the slab sums add in a different order from the undecomposed
    grid's, so the integrals agree to rounding, not bit for bit."""
    out = dict(parts[0])
    for k in _SUMMED:
        out[k] = type(parts[0][k])(sum(p[k] for p in parts))
    out["divb_max"] = max(p["divb_max"] for p in parts)
    out["PhiB"] = out["phib"] / math.sqrt(abs(out["mdot"])) if out["mdot"] != 0.0 else 0.0
    out["eta"] = (out["edot"] - out["mdot"]) / abs(out["mdot"]) if out["mdot"] != 0.0 else 0.0
    out["disk_mass"] = out["disk_eb"] = 0.0  # set by the torus setup only
    return out


def _bary(parts):
    num = sum(p[0] for p in parts)
    den = sum(p[1] for p in parts)
    return (num / den if den > 0.0 else 0.0), den, num


def _stream_of(engine):
    s = getattr(engine, "stream", None)
    return torch.cuda.stream(s) if s is not None else contextlib.nullcontext()


class SlabRing:
    """All slabs of one grid on one device, in phi order, sharing one stream."""

    def __init__(self, engines):
        self.e = list(engines)
        e0 = self.e[0]
        self.lo = [torch.empty(e.plane_numel, dtype=e.dtype, device=e.device) for e in self.e]
        self.hi = [torch.empty(e.plane_numel, dtype=e.dtype, device=e.device) for e in self.e]
        self.dtd_buf = torch.empty(3, dtype=torch.float64, device=e0.device)

    @classmethod
    def create(cls, grid: G.GridParams, phys: G.PhysParams, R: int, a: float, stream=None):
        stream = stream or torch.cuda.Stream(device=grid.device)
        sg = slab_grid(grid, R)
        return cls([CtxSlab.create(sg, phys, a, stream) for _ in range(R)])

    def set_state(self, P, U, t, dt):
        """P, U: the whole grid's state (host arrays or device tensors)."""
        R = len(self.e)
        for r, e in enumerate(self.e):
            with _stream_of(e):  # a device slice is copied on the slab's stream
                e.set_state(split_phi(P, R, r), split_phi(U, R, r), t, dt)
        self.exchange(0)

    def exchange(self, which):
        R = len(self.e)
        for r, e in enumerate(self.e):
            e.pack(which, 0, self.lo[r])
            e.pack(which, 1, self.hi[r])
        for r, e in enumerate(self.e):
            e.unpack(which, 0, self.hi[(r - 1) % R])
            e.unpack(which, 1, self.lo[(r + 1) % R])

    def step(self, nsteps=1):
        for _ in range(nsteps):
            for r, e in enumerate(self.e):
                e.stage(0)
                e.dtd(self.dtd_buf, accumulate=r > 0)
            self.exchange(1)
            for e in self.e:
                e.stage(1)
            self.exchange(0)
            for e in self.e:
                e.finish(self.dtd_buf)

    def diagnostics(self):
        return combine_diagnostics([e.diagnostics() for e in self.e])

    def barycentric_radius(self, r_bar_max=80.0):
        """(<r>, mass, numerator) of Eq. 43 over the whole grid: the slabs'
        sums added in slab order."""
        return _bary([e.barycentric_sums(r_bar_max) for e in self.e])

    def close(self):
        for e in self.e:
            e.close()


class SlabRank:
    """This process's slab of a grid split over the ranks of a process group,
    rank r owning phi slab r.  Ghost planes travel by send/recv (tagged by
    direction and posted in the same order on every rank, so that two ranks
    that are each other's left and right neighbours still match them); the
    CFL minima are combined by a MIN all-reduce."""

    TAG_RIGHTWARD, TAG_LEFTWARD = 1, 2

    def __init__(self, engine, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.e = engine
        self.rank = dist.get_rank(group)
        self.R = dist.get_world_size(group)
        self.left, self.right = (self.rank - 1) % self.R, (self.rank + 1) % self.R
        if group is not None:
            self.left = dist.get_global_rank(group, self.left)
            self.right = dist.get_global_rank(group, self.right)
        mk = lambda: torch.empty(engine.plane_numel, dtype=engine.dtype, device=engine.device)
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(), mk(), mk(), mk()
        self.dtd_buf = torch.empty(3, dtype=torch.float64, device=engine.device)

    def set_state(self, P, U, t, dt):
        """P, U: the whole grid's state (every rank holds the same); this
        rank keeps its slab."""
        with _stream_of(self.e):
            self.e.set_state(split_phi(P, self.R, self.rank), split_phi(U, self.R, self.rank), t, dt)
        self.exchange(0)

    def exchange(self, which):
        e, dist = self.e, self.dist
        e.pack(which, 0, self.send_lo)
        e.pack(which, 1, self.send_hi)
        if self.R == 1:
            e.unpack(which, 0, self.send_hi)
            e.unpack(which, 1, self.send_lo)
            return
        with _stream_of(e):
            ops = [dist.P2POp(dist.isend, self.send_hi, self.right, self.group, self.TAG_RIGHTWARD),
                   dist.P2POp(dist.isend, self.send_lo, self.left, self.group, self.TAG_LEFTWARD),
                   dist.P2POp(dist.irecv, self.recv_lo, self.left, self.group, self.TAG_RIGHTWARD),
                   dist.P2POp(dist.irecv, self.recv_hi, self.right, self.group, self.TAG_LEFTWARD)]
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        e.unpack(which, 0, self.recv_lo)
        e.unpack(which, 1, self.recv_hi)

    def step(self, nsteps=1):
        e = self.e
        for _ in range(nsteps):
            e.stage(0)
            e.dtd(self.dtd_buf)
            self.exchange(1)
            e.stage(1)
            self.exchange(0)
            if self.R > 1:
                with _stream_of(e):
                    self.dist.all_reduce(self.dtd_buf, op=self.dist.ReduceOp.MIN, group=self.group)
            e.finish(self.dtd_buf)

    def diagnostics(self):
        """The whole grid's diagnostics on every rank (combine_diagnostics
        over all ranks' slabs, gathered on the host)."""
        parts = [None] * self.R
        self.dist.all_gather_object(parts, self.e.diagnostics(), group=self.group)
        return combine_diagnostics(parts)

    def barycentric_radius(self, r_bar_max=80.0):
        parts = [None] * self.R
        self.dist.all_gather_object(parts, self.e.barycentric_sums(r_bar_max), group=self.group)
        return _bary(parts)


__all__ = ["NG", "slab_grid", "split_phi", "combine_diagnostics", "CtxSlab", "SlabRing", "SlabRank"]
